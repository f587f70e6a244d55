"""Brute-force enumeration of random-walk path probabilities, written
directly from Eq. (prob), Eq. (node2vec) and the MetaPath rule (Sec. 2.1) on
adjacency sets; shared by the oracle pins and the GPU walk tests."""
import numpy as np
from scipy import stats


def _bf_weight(adj, h, lab, v, u, vprev, hop, algo, p, q, schema, gamma=0.2):
    hv = h[(v, u)]
    if algo == "pagerank2":  # Eq. (2ndpr); u = v' takes the "otherwise" branch, hop 0 is first-order
        if vprev is None:
            return hv
        dv, dp = len(adj[v]), len(adj[vprev])
        md = max(dv, dp)
        if u in adj[vprev]:
            return hv * ((1 - gamma) / dv + gamma / dp) * md
        return hv * ((1 - gamma) / dv) * md
    if algo == "weighted":
        return hv
    if algo == "node2vec":
        if vprev is None:
            return hv
        if u == vprev:
            return hv / p
        if u in adj[vprev]:
            return hv
        return hv / q
    return hv if lab[(v, u)] == schema[hop % len(schema)] else 0.0


def bf_paths(g, start, length, algo, p, q, schema, gamma=0.2):
    """{path tuple (padded with -1 after a dead end): probability}."""
    n = g.n
    adj = [set(g.cols[g.offsets[i]:g.offsets[i + 1]].tolist()) for i in range(n)]
    h, lab = {}, {}
    for v in range(n):
        for k in range(g.offsets[v], g.offsets[v + 1]):
            u = int(g.cols[k])
            h[(v, u)] = float(g.h[k]) if g.h is not None else 1.0
            lab[(v, u)] = int(g.labels[k]) if g.labels is not None else 0
    out = {}

    def rec(path, prob):
        hop = len(path) - 1
        if hop == length:
            out[tuple(path)] = out.get(tuple(path), 0.0) + prob
            return
        v = path[-1]
        vprev = path[-2] if len(path) > 1 else None
        ws = {u: _bf_weight(adj, h, lab, v, u, vprev, hop, algo, p, q, schema, gamma) for u in sorted(adj[v])}
        tot = sum(ws.values())
        if tot <= 0:
            padded = tuple(path) + (-1,) * (length - hop)
            out[padded] = out.get(padded, 0.0) + prob
            return
        for u, w in ws.items():
            if w > 0:
                rec(path + [u], prob * w / tot)

    rec([start], 1.0)
    return out


def merged_chisquare(bf, rows):
    """Chi-square p-value of sampled rows (int array [W][L+1]) against the
    path probabilities `bf`, merging bins of expected count < 5.  Fails if a
    row has probability zero."""
    keys = list(bf.keys())
    index = {k: i for i, k in enumerate(keys)}
    counts = np.zeros(len(keys))
    for row in map(tuple, np.asarray(rows).tolist()):
        assert row in index, f"walk {row} has probability zero"
        counts[index[row]] += 1
    exp = np.array([bf[k] for k in keys]) * len(rows)
    order = np.argsort(exp)
    obs_m, exp_m, acc_o, acc_e = [], [], 0.0, 0.0
    for i in order:
        acc_o += counts[i]
        acc_e += exp[i]
        if acc_e >= 5:
            obs_m.append(acc_o)
            exp_m.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0:
        obs_m[-1] += acc_o
        exp_m[-1] += acc_e
    return float(stats.chisquare(obs_m, exp_m).pvalue)
