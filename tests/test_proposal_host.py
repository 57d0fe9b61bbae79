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
