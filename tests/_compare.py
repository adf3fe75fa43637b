"""Comparison rules of the parity tests (GPU results vs the FP64 oracle).

Scores: |Q_gpu - Q_ref| <= REL * max(|Q_ref|, 1e-3 |Q_ref,top1|) with REL = 1e-5.
Indices and shifts: identical, except at a near-tie, where the oracle's own Q for the
GPU's choice lies within the same tolerance of the oracle's value at that rank (several
answers are then correct; what is unique -- the ranked scores -- is still compared).
"""
from __future__ import annotations

import numpy as np

REL = 1e-5


def tol(q_ref, q_top):
    return REL * np.maximum(np.abs(q_ref), 1e-3 * np.abs(q_top))


def template_q_all(P: np.ndarray, lib, k: int) -> np.ndarray:
    """Oracle Q(k, s) for all shifts of one template on one polar image (Eq. 1 written out)."""
    n_theta = lib.n_theta
    nP = float(np.sqrt(np.sum(P * P)))
    d = nP * lib.norm[k]
    q = np.zeros(n_theta)
    if d <= 0:
        return q
    for i in range(lib.off[k], lib.off[k + 1]):
        q += lib.I[i] * np.roll(P[lib.ri[i]], -int(lib.ti[i]))
    return q / d


def compare_hits(hits: np.ndarray, ref: dict, lib, patterns=None) -> dict:
    """hits: structured [n][N] (tmgb.HIT_DTYPE) for the same patterns as ref (oracle.index).
    Raises AssertionError on a violation; returns counts of exact matches and near-ties."""
    n, N = hits.shape
    idx = range(n) if patterns is None else patterns
    stats = dict(patterns=0, exact=0, near_tie_template=0, near_tie_shift=0, top1_same=0)
    for p in idx:
        stats["patterns"] += 1
        rk, rs, rq = ref["template"][p], ref["shift"][p], ref["score"][p]
        q_top = rq[0] if np.isfinite(rq[0]) else 1.0
        gk = hits["template_index"][p].astype(np.int64)
        gs = hits["shift"][p].astype(np.int64)
        gq = hits["score"][p].astype(np.float64)
        # GPU rows are valid: sorted by (score desc, template asc), distinct templates
        valid = gk >= 0
        assert np.array_equal(valid, rk >= 0), f"pattern {p}: padding differs {gk} vs {rk}"
        v = int(valid.sum())
        assert len(set(gk[:v].tolist())) == v, f"pattern {p}: repeated template {gk}"
        for j in range(v - 1):
            assert gq[j] > gq[j + 1] or (gq[j] == gq[j + 1] and gk[j] < gk[j + 1]), f"pattern {p}: order {gq} {gk}"
        assert np.all(np.isneginf(gq[v:])), f"pattern {p}: padding score {gq}"
        all_exact = True
        for j in range(v):
            t = tol(rq[j], q_top)
            assert abs(gq[j] - rq[j]) <= t, f"pattern {p} rank {j}: Q {gq[j]} vs {rq[j]} (tol {t})"
            if gk[j] != rk[j]:
                qg = ref["q_best"][p, gk[j]]
                assert abs(qg - rq[j]) <= t, (f"pattern {p} rank {j}: template {gk[j]} (oracle Q {qg}) "
                                              f"vs {rk[j]} (Q {rq[j]}) not a near-tie")
                stats["near_tie_template"] += 1
                all_exact = False
                # its shift must attain its own best within tolerance
                qa = template_q_all(ref["polar"][p], lib, int(gk[j]))
                assert abs(qa[gs[j]] - qg) <= t, f"pattern {p} rank {j}: shift {gs[j]} not a best shift"
            elif gs[j] != rs[j]:
                qa = template_q_all(ref["polar"][p], lib, int(gk[j]))
                assert abs(qa[gs[j]] - rq[j]) <= t, (f"pattern {p} rank {j}: shift {gs[j]} (Q {qa[gs[j]]}) vs "
                                                     f"{rs[j]} (Q {rq[j]}) not a near-tie")
                stats["near_tie_shift"] += 1
                all_exact = False
        stats["exact"] += int(all_exact)
        stats["top1_same"] += int(v == 0 or (gk[0] == rk[0] and gs[0] == rs[0]))
    return stats


def compare_scores(q_gpu, s_gpu, ref_q, ref_s, P_ref, lib, patterns=None) -> dict:
    """Per-(pattern, template) best Q and shift (the correlate stage)."""
    n, K = ref_q.shape
    idx = range(n) if patterns is None else patterns
    near = 0
    for p in idx:
        act = np.isfinite(ref_q[p])
        assert np.array_equal(np.isfinite(q_gpu[p]), act), f"pattern {p}: masked sets differ"
        q_top = np.max(ref_q[p][act]) if act.any() else 1.0
        t = tol(ref_q[p][act], q_top)
        d = np.abs(q_gpu[p][act].astype(np.float64) - ref_q[p][act])
        bad = np.flatnonzero(d > t)
        assert bad.size == 0, f"pattern {p}: {bad.size} Q outside tolerance, worst {d.max()} (tol {t[bad[0]]})"
        ks = np.flatnonzero(act & (s_gpu[p] != ref_s[p]))
        for k in ks:
            qa = template_q_all(P_ref[p], lib, int(k))
            assert abs(qa[s_gpu[p, k]] - ref_q[p, k]) <= tol(ref_q[p, k], q_top), \
                f"pattern {p} template {k}: shift {s_gpu[p, k]} vs {ref_s[p, k]} not a near-tie"
            near += 1
        assert np.all(s_gpu[p][~act] == -1)
    return dict(near_tie_shift=near)
