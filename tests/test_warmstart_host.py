"""On the CPU: the oracle's warm-start normalisations (oracle/warmstart.py: the feature
standardisation and the per-order output scale, against hand-worked values), which gs_ws_normalise
is checked against on the GPU, and the driver's parameter packing that gs_mlp_set_params reads.
No GPU, no kernels."""
import math

import numpy as np

from oracle.warmstart import N_IN, order_scale, standardisation
from paper_1412_7466_gb300.warmstart import pack


def test_standardisation_sweep_columns_and_constants():
    rng = np.random.default_rng(3)
    X0 = rng.standard_normal((500, N_IN)) * 3.0 + 1.5
    X0[:, 20] = 7.0                                   # a constant feature
    mu, sd = standardisation(X0, (-2.0, -1.0), (30.0, 50.0))
    # theta (column 10) and k1 (column 11): the sweep's uniform ranges, not the sample
    assert mu[10] == -1.5 and math.isclose(sd[10], 1.0 / math.sqrt(12.0))
    assert mu[11] == 40.0 and math.isclose(sd[11], 20.0 / math.sqrt(12.0))
    # a constant column keeps its mean and gets unit spread (no division by zero)
    assert mu[20] == 7.0 and sd[20] == 1.0
    # the rest are the sample moments
    others = [c for c in range(N_IN) if c not in (10, 11, 20)]
    np.testing.assert_allclose(mu[others], X0[:, others].mean(0))
    np.testing.assert_allclose(sd[others], X0[:, others].std(0))


def test_order_scale_keeps_orders_by_share_of_beta():
    # rms target t_n = sqrt(ms_t); share of beta = rms(s_n t_n) = sqrt(ms_st)
    ms_t = np.array([4.0, 1.0, 9.0, 1.0, 0.25])
    ms_st = np.array([1.0, 1e-9, 4.0, 1e-7, 0.0])    # shares 1, 3.2e-5, 2, 3.2e-4, 0 (top 2)
    sc = order_scale(ms_t, ms_st, share=1e-4)
    # kept where share > 1e-4 * 2: orders 0, 2, 3 -> their rms target; the others are not predicted
    np.testing.assert_array_equal(sc, [2.0, 0.0, 3.0, 1.0, 0.0])


def test_order_scale_degenerate_inputs():
    assert np.all(order_scale(np.zeros(5), np.zeros(5)) == 0.0)            # nothing to predict
    sc = order_scale(np.array([1.0, np.inf, 4.0]), np.array([1.0, 1.0, 1.0]))
    np.testing.assert_array_equal(sc, [1.0, 0.0, 2.0])                      # non-finite target dropped
    sc = order_scale(np.array([1.0, 0.0]), np.array([1.0, 1.0]))
    np.testing.assert_array_equal(sc, [1.0, 0.0])                           # zero target dropped


def test_pack_layout():
    w = np.arange(10, dtype=np.float64)
    mu, sd, sc = np.full(N_IN, 0.5), np.full(N_IN, 2.0), np.array([1.0, 0.0, 3.0])
    v = pack(w, mu, sd, sc)
    assert v.dtype == np.float32 and v.shape == (10 + 2 * N_IN + 3,)
    np.testing.assert_array_equal(v[:10], w)
    np.testing.assert_array_equal(v[10:10 + N_IN], mu)
    np.testing.assert_array_equal(v[10 + N_IN:10 + 2 * N_IN], sd)
    np.testing.assert_array_equal(v[-3:], sc)
