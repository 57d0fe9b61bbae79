"""Host helpers of the learned proposal (C ABI, no GPU work) against the
FP64 reference: region targets and the proposed period set."""

import numpy as np

from oracle import cnn


def test_region_targets_and_proposal_match_the_reference():
    import paper_2607_00348_gb300 as pkg
    rng = np.random.default_rng(0)
    periods = np.sort(np.exp(rng.uniform(np.log(0.45), np.log(1100.0), 20000)))
    sr = rng.uniform(size=periods.size)
    tgt, mask = pkg.region_targets(periods, sr)
    t_or, m_or = cnn.region_targets(periods, sr)
    np.testing.assert_array_equal(mask, m_or.astype(np.float32))
    np.testing.assert_array_equal(tgt, t_or.astype(np.float32))
    for frac in (0.05, 0.2, 1.0):
        scores = rng.uniform(size=cnn.N_REG).astype(np.float32)
        scores[5] = scores[9]                      # a tie: the lower region first
        got = pkg.proposal_periods(periods, scores, frac)
        want = cnn.proposed_periods(periods, scores.astype(np.float64), m_or, frac)
        np.testing.assert_array_equal(got, want)


def test_library_parameter_layout_matches_the_reference():
    import paper_2607_00348_gb300 as pkg
    from paper_2607_00348_gb300 import proposal as pr
    n = sum(int(np.prod(s)) for _, s in cnn.param_shapes())
    assert pkg.gtls.load().gtls_cnn_param_count() == n == pr.init_params(0).size


def test_triage_threshold_keeps_every_calibration_detection():
    # brute force over a synthetic evaluation record: the threshold of each
    # half is the smallest score of its plain detections, the other half is
    # searched where its score reaches it, and the rates follow
    from paper_2607_00348_gb300 import proposal as pr
    rng = np.random.default_rng(3)
    n = 40
    per = []
    for i in range(n):
        inj = rng.uniform() < 0.5
        det = bool(inj and rng.uniform() < 0.7)
        per.append({"score_max": float(rng.uniform(0.3, 1.0) if det else rng.uniform(0.0, 0.8)),
                    "plain_detected": det, "inj_period": 3.0 if inj else None})
    rows = pr.triage(per, 1000.0)
    assert len(rows) == 2
    halves = (range(0, n // 2), range(n // 2, n))
    for row, (cal, test) in zip(rows, ((halves[0], halves[1]), (halves[1], halves[0]))):
        thr = min(per[i]["score_max"] for i in cal if per[i]["plain_detected"])
        assert row["threshold"] == thr
        keep = [i for i in test if per[i]["score_max"] >= thr]
        assert row["searched"] == len(keep) and row["curves"] == len(test)
        assert row["detections_kept"] == sum(per[i]["plain_detected"] for i in keep)
        assert row["detections_plain"] == sum(per[i]["plain_detected"] for i in test)
        n_inj = sum(per[i]["inj_period"] is not None for i in test)
        assert row["recall"] == row["detections_kept"] / n_inj
        assert abs(row["lc_per_hour"] - 1000.0 * len(test) / len(keep)) < 1e-9


def test_triage_threshold_of_the_stored_evaluation():
    # the bench's learned leg reads the smaller cross-validated threshold
    import json
    import os
    from paper_2607_00348_gb300 import proposal as pr
    path = os.path.join(os.path.dirname(pr.WEIGHTS), "proposal_eval.json")
    with open(path) as f:
        rows = json.load(f)["triage"]
    assert pr.triage_threshold() == min(r["threshold"] for r in rows)
    assert all(r["detections_kept"] <= r["detections_plain"] for r in rows)
