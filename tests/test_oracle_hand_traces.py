"""Hand-traced pins of the oracle's two decision sequences.

Algorithm 1 (Sec. 5) with recomputes: tests/golden/aps_trace.json holds two
small 2-D cases worked by hand from the circular-segment cap, with rho, p and
r after every step.  The L2 case fires two recomputes that move the stop
point; the inner-product case has rho grow after a scan, so a recompute that
only looks at shrinking radii stops early.  A dropped recompute, a rho that is
never updated, p_0 kept from before a recompute, or r summed from stale p each
change the scan sequence or the final r.

Merge verify (Sec. 4 "Exact Merge Delta", Stage 2): tests/golden/merge_verify.json
is one cold partition whose rows go to three receivers, with each receiver's
Delta s_m, Delta A_m and Eq. 5 worked out with exact fractions, once where the
merge commits and once where the exact delta rejects what the estimate
accepted.
"""

import json
import os

import numpy as np
import pytest

from oracle import aps, kmeans, knn, maintenance

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


APS_CASES = _load("aps_trace.json")["cases"]


def _level(case):
    C = np.array(case["centroids"], np.float32)
    V = [np.array([r["x"] for r in rows], np.float32).reshape(-1, 2) for rows in case["partitions"]]
    I = [np.array([r["id"] for r in rows], np.int64) for rows in case["partitions"]]
    return kmeans.Level(C, V, I)


@pytest.mark.parametrize("case", APS_CASES, ids=[c["name"] for c in APS_CASES])
def test_algorithm1_reproduces_the_hand_trace(case):
    lv = _level(case)
    q = np.array(case["q"], np.float64)
    metric = knn.L2 if case["metric"] == "l2" else knn.IP
    prm = aps.Params(k=case["k"], recall_target=case["recall_target"], f_M=(1.0,), tau_rho=case["tau_rho"],
                     beta_mode="exact")
    cand, cD = aps.root_candidates(q, lv, 1.0)
    assert [int(c) for c in cand] == case["candidate_order"]
    t = aps.bisector_distances(cD, lv.centroids[cand])
    # coordinates are stored in FP32, the hand trace used their decimal values
    np.testing.assert_allclose(t, case["t"], rtol=1e-6, atol=1e-7)
    res = aps.aps_level(q, lv, list(cand), cD, case["k"], case["recall_target"], prm, 2, metric, None)
    assert [int(cand[p]) for p in res["scanned"]] == case["scan_sequence"]
    assert len(res["steps"]) == len(case["steps"])
    for got, want in zip(res["steps"], case["steps"]):
        assert got["pos"] == want["scanned_position"]
        assert got["recomputed"] == want["recomputed"]
        assert got["rho"] == pytest.approx(want["rho"], rel=1e-6)
        np.testing.assert_allclose(got["p"], want["p"], rtol=1e-5, atol=1e-7)
        assert got["r"] == pytest.approx(want["r"], rel=1e-6)
    assert res["r"] == pytest.approx(case["final_r"], rel=1e-6)
    # the whole search (root scoring, Algorithm 1) ends the same way
    out = aps.search([lv], q[None, :], prm, metric=metric)
    assert int(out["nprobe"][0]) == case["nprobe"]
    assert out["scanned"][0][0] == case["scan_sequence"]
    assert float(out["r"][0]) == pytest.approx(case["final_r"], rel=1e-6)


def test_hand_traces_exercise_recomputes_both_ways():
    """The golden cases cover what they claim: two recomputes and a step
    without one (L2), and a recompute on a growing radius (IP)."""
    l2, ip = APS_CASES
    rec = [s["recomputed"] for s in l2["steps"][1:]]
    assert rec.count(True) >= 2 and rec.count(False) >= 1
    grew = [b["rho"] > a["rho"] and b["recomputed"] for a, b in zip(ip["steps"], ip["steps"][1:])]
    assert any(grew)


MERGE = _load("merge_verify.json")


def _merge_level():
    C, V, I = [], [], []
    for p in MERGE["partitions"]:
        c = np.array(p["centroid"], np.float64)
        if "rows" in p:
            rows = np.array(p["rows"], np.float64)
        else:
            i = np.arange(p["size"])
            rows = c[None, :] + np.stack([0.1 * (i % 5) - 0.2, 0.1 * (i // 5) - 0.15], axis=1)
        C.append(c)
        V.append(rows.astype(np.float32))
        I.append(p["first_id"] + np.arange(rows.shape[0], dtype=np.int64))
    return kmeans.Level(np.array(C, np.float32), V, I)


@pytest.mark.parametrize("case", MERGE["cases"], ids=["commit", "reject"])
def test_merge_verify_hand_case(case):
    lv = _merge_level()
    names = [p["name"] for p in MERGE["partitions"]]
    A = [case["A"][n] for n in names]
    pts = np.array(MERGE["lambda_points"], np.float64)
    prm = maintenance.MaintParams(maintenance.Latency(pts[:, 0], pts[:, 1]), tau=MERGE["tau"],
                                  alpha=MERGE["alpha"], refine_radius=MERGE["refine_radius"],
                                  s_min=MERGE["s_min"], refine=False)
    before = [(c.copy(), v.copy(), i.copy()) for c, v, i in zip(lv.centroids, lv.vectors, lv.ids)]
    detail = []
    log, keep = maintenance.maintain_level(lv, A, prm, 0, detail=detail)
    # the only candidate is the merge of j (index 3); nothing is split
    assert [(k, j) for k, j, *_ in log] == [("merge", 3)]
    (dt,) = detail
    assert dt["estimate"] == pytest.approx(case["estimate"], abs=1e-12)
    assert dt["delta"] == pytest.approx(case["delta"], abs=1e-12)
    assert dt["ok"] is case["commit"]
    want = MERGE["nearest_remaining"]["delta_s"]
    got = {names[m]: v for m, v in dt["receivers"].items()}
    assert sorted(got) == ["a", "b", "c"]
    for n in "abc":
        ds, dA = got[n]
        assert ds == want[n]
        assert dA == pytest.approx(case["delta_A"][n], abs=1e-15)
    # Eq. 5 term by term from the recorded receivers
    lam = prm.lam
    sizes = {n: lv_size for n, lv_size in zip(names, [20, 30, 40, 7])}
    for n in "abc":
        ds, dA = got[n]
        term = (case["A"][n] + dA) * lam(sizes[n] + ds) - case["A"][n] * lam(sizes[n])
        assert term == pytest.approx(case["receiver_terms"][n], abs=1e-12)
    assert sorted(v.shape[0] for v in lv.vectors) == sorted(case["sizes_after"])
    if case["commit"]:
        assert keep == [0, 1, 2]
        j_ids = set(range(300, 307))
        moved = {names[m]: len(j_ids & set(lv.ids[m].tolist())) for m in range(3)}
        assert moved == want
    else:
        assert keep == [0, 1, 2, 3]
        for (c0, v0, i0), c1, v1, i1 in zip(before, lv.centroids, lv.vectors, lv.ids):
            assert np.array_equal(c0, c1) and np.array_equal(v0, v1) and np.array_equal(i0, i1)
