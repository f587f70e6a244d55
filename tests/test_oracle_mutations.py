"""Mutation check of the oracle's pins (CPU only).

Each case plants one plausible mistake in a copy of ``oracle/fw_oracle.c``
(a swapped parameter, a wrong index, a dropped term, a flipped comparison,
a wrong constant), compiles the copy, and runs the pins of
``tests/test_oracle.py`` against it in a child process: at least one pin must
fail.  The unmodified source, built the same way, must pass them all, so a
mutant's failure comes from the planted mistake and not from the harness.

Mistakes that leave every probability unchanged in exact arithmetic (the
max_d factor of Eq. (2ndpr) scales w1 and w2 alike; the hop-0 weight of
node2vec is the same for every neighbour) are not listed: only the bit-exact
GPU parity tests can tell those apart.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "fw_oracle.c")

# name -> (text in fw_oracle.c, replacement)
MUTANTS = {
    # Philox4x32-10 (Salmon et al.): the second Weyl key increment
    "philox_key_weyl": ("k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;"),
    # exact-mode uniform: which output word, and the 24-bit grid
    "uniform_word": ("(float)(x[0] >> 8)", "(float)(x[1] >> 8)"),
    "uniform_shift": ("(float)(x[0] >> 8)", "(float)(x[0] >> 9)"),
    # Eq. (node2vec): 1/p and 1/q exchanged
    "node2vec_swap_pq": ("const float inv_p = or_recip(p), inv_q = or_recip(q);",
                         "const float inv_p = or_recip(q), inv_q = or_recip(p);"),
    # Eq. (node2vec): membership tested in N(v) instead of N(v')
    "node2vec_wrong_row": ("else if (is_neighbour(offsets, cols, vprev, u)) w = 1.0f;",
                           "else if (is_neighbour(offsets, cols, v, u)) w = 1.0f;"),
    # Eq. (node2vec): the return edge not recognised
    "node2vec_no_return": ("else if (u == vprev) w = inv_p;", "else if (u == vprev + 1) w = inv_p;"),
    # Eq. (prob): the property weight h dropped
    "prob_drop_h": ("wt[k] = w * hk;", "wt[k] = w;"),
    # MetaPath rule: schema index shifted by one hop
    "metapath_schema_shift": ("schema[step % schema_len]", "schema[(step + 1) % schema_len]"),
    # MetaPath rule: filter inverted
    "metapath_filter_inverted": ("(labels[s + k] == schema[step % schema_len])",
                                 "(labels[s + k] != schema[step % schema_len])"),
    # Eq. (2ndpr): the two weights exchanged
    "pagerank2_swap_weights": ("? pr_w1 : pr_w2;", "? pr_w2 : pr_w1;"),
    # Eq. (2ndpr): gamma / d(v) instead of gamma / d(v')
    "pagerank2_wrong_degree": ("const float t2 = gamma / dp;", "const float t2 = gamma / dv;"),
    # ITS (Sec. 2.2): strict comparison made inclusive
    "icdf_inclusive": ("if (t < run) return k;", "if (t <= run) return k;"),
    # walk: the previous node never advances
    "walk_prev_stuck": ("        prev = cur;\n        cur = nxt;", "        cur = nxt;"),
    # Sec. 4.2 preprocessing: minimum instead of maximum
    "node_stats_min": ("if (x > m) m = x;", "if (x < m || m == 0.0f) m = x;"),
    # Sec. 3.3 bound: 1/p left out of max(w)
    "bound_drop_inv_p": ("wmax = ip > 1.0f ? ip : 1.0f;", "wmax = 1.0f;"),
    # Eq. (sum_estimation): mean over two values instead of three
    "sum_estimate_mean": ("wmean = (float)(((double)ip + 1.0 + (double)iq) / 3.0);",
                          "wmean = (float)(((double)ip + 1.0 + (double)iq) / 2.0);"),
    # Eq. (runtime): the comparison reversed
    "cost_model_reversed": ("return (r * B < S) ? OR_MODE_RJS : OR_MODE_RVS;",
                            "return (r * B > S) ? OR_MODE_RJS : OR_MODE_RVS;"),
    # per-label statistics: label sums into the wrong slot
    "label_stats_slot": ("lsum[v * 8 + l] += (double)x;", "lsum[v * 8 + (l + 1) % 8] += (double)x;"),
    # Eq. (prob): weights returned without normalisation
    "probs_not_normalised": ("probs[k] = total > 0.0 ? (double)wt[k] / total : 0.0;",
                             "probs[k] = total > 0.0 ? (double)wt[k] : 0.0;"),
    # walk: the row after a dead end filled with node 0 instead of -1
    "walk_suffix_zero": ("for (int32_t r = j + 1; r <= len; ++r) row[r] = -1;",
                         "for (int32_t r = j + 1; r <= len; ++r) row[r] = 0;"),
    # walk: the random-stream id ignores walker_base
    "walk_base_ignored": ("const uint32_t wid = ids ? ids[i] : walker_base + (uint32_t)i;",
                          "const uint32_t wid = ids ? ids[i] : (uint32_t)i;"),
    # per-label statistics: the last weight instead of the largest
    "label_stats_last": ("if (x > lmax[v * 8 + l]) lmax[v * 8 + l] = x;", "lmax[v * 8 + l] = x;"),
    # 8-bit weights: codes allowed to reach 0 (an edge losing its weight)
    "quantize_clamp_zero": ("if (c < 1.0f) c = 1.0f;", "if (c < 0.0f) c = 0.0f;"),
    # 8-bit weights: truncation instead of round-to-nearest
    "quantize_truncate": ("float c = rintf(h[i] / s);", "float c = floorf(h[i] / s);"),
    # 8-bit codes: the scale off by one code, or taken from every row instead of the node's own
    "quantize_scale_256": ("const float s = row_max / 255.0f;", "const float s = row_max / 256.0f;"),
    "quantize_global_max": ("for (int64_t i = offsets[v]; i < offsets[v + 1]; ++i)\n      if (h[i] > row_max)",
                            "for (int64_t i = 0; i < offsets[n]; ++i)\n      if (h[i] > row_max)"),
    # RJS (Sec. 3.3): the proposal taken from the word that also gives U
    "rjs_index_word": ("lemire_index(x[0], slots, &sl) && !lemire_index(x[1], slots, &sl)) continue;\n    int64_t k",
                       "lemire_index(x[2], slots, &sl) && !lemire_index(x[1], slots, &sl)) continue;\n    int64_t k"),
    # RJS: the index taken as x mod d instead of Lemire's multiply-shift
    "rjs_index_modulo": ("*k = (uint32_t)(m >> 32);", "*k = x % d;"),
    # RJS: the bound from the row's first weight instead of h_MAX[v]
    "rjs_bound_first_h": ("if (x > hmax) hmax = x;", "if (hmax == 0.0f) hmax = x;"),
    # weight-class envelope: an entry at exactly h_MAX/2 put into class 0
    "rjs_class_boundary": ("const int ck = hrow[k] > half ? 0", "const int ck = hrow[k] >= half ? 0"),
    # weight-class envelope: class 1 proposed twice as often as class 2 but bounded by B
    "rjs_class_bound": ("        bound = 0.5f * B;", "        bound = B;"),
    # label-segment envelope: an entry at exactly M/2^(c+1) moved up a class
    "rjs_label_class_boundary": ("while (ck < 4 && !(x > t))", "while (ck < 4 && !(x >= t))"),
    # label-segment envelope: class bounds quartered instead of halved
    "rjs_label_bound": ("      bound = 0.5f * bound;", "      bound = 0.25f * bound;"),
    # RJS: acceptance test reversed
    "rjs_accept_reversed": ("if (U * bound < wt[k]) return k;", "if (U * bound > wt[k]) return k;"),
}


def _build(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", *oracle.CFLAGS, str(src), "-o", str(so), "-lm"], check=True, capture_output=True)
    return str(so)


def _run_pins(so):
    env = dict(os.environ, FW_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle.py"), "-x", "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    return r.returncode, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """(return code, output tail) of the pins for the unmodified copy and for
    every mutant; the child runs proceed side by side."""
    with open(SRC) as f:
        text = f.read()
    d = tmp_path_factory.mktemp("mutants")
    sources = {"unmodified": text}
    for name, (old, new) in MUTANTS.items():
        if text.count(old) == 1:
            sources[name] = text.replace(old, new)
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {name: ex.submit(lambda nm, src: _run_pins(_build(d, nm, src)), name, src)
                for name, src in sources.items()}
        return {name: f.result() for name, f in futs.items()}


def test_unmodified_oracle_passes_through_the_harness(outcomes):
    rc, out = outcomes["unmodified"]
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(outcomes, name):
    old, _ = MUTANTS[name]
    with open(SRC) as f:
        assert f.read().count(old) == 1, f"{name}: the text to mutate must occur exactly once"
    rc, out = outcomes[name]
    # 1 = some test failed; anything else (0 = all passed, 2+ = harness or
    # collection error) does not show that a pin caught the mistake
    assert rc == 1, f"{name}: pins returned {rc}\n{out}"
    assert " failed" in out, out
