"""The seeded input generators shared by the oracle and the CUDA path (workloads/): reproducible,
and producing the structures their docstrings state — non-overlapping disks under the periodic
minimum image, inside the middle layer's strip; Wood angles where kappa_n = k1 (Sec. 2); the
batched angle list containing that angle exactly; uneven geometry sizes; the network's parameter
layout.  CPU only."""
import math

import numpy as np
import pytest

import workloads as W


def _min_image_dist2(xy, d=1.0):
    dx = np.abs(xy[:, None, 0] - xy[None, :, 0])
    dx = np.minimum(dx, d - dx)
    dy = xy[:, None, 1] - xy[None, :, 1]
    r2 = dx * dx + dy * dy
    np.fill_diagonal(r2, np.inf)
    return r2


@pytest.mark.parametrize("M,r,gap", [(10, 0.04, 0.02), (1000, 0.008, 0.004)])
def test_disks_reproducible_non_overlapping_inside_strip(M, r, gap):
    a = W.disks(M, r, gap, 2.0, 40.0, seed=7, p=12)
    b = W.disks(M, r, gap, 2.0, 40.0, seed=7, p=12)
    np.testing.assert_array_equal(a["xy"], b["xy"])
    c = W.disks(M, r, gap, 2.0, 40.0, seed=8, p=12)
    assert not np.array_equal(a["xy"], c["xy"])
    xy = a["xy"]
    assert xy.shape == (M, 2) and a["radius"].shape == (M,) and a["kp"].shape == (M,)
    assert np.all(a["radius"] == r) and np.all(a["kp"] == 80.0) and a["p"] == 12
    # brute force: every pair at least 2r + gap apart under the minimum image in x
    assert np.sqrt(_min_image_dist2(xy).min()) >= 2 * r + gap - 1e-15
    # centres in one period and inside the strip |y| < min(0.4, 0.45 - 0.04 - r)
    assert np.all(xy[:, 0] >= -0.5) and np.all(xy[:, 0] < 0.5)
    assert np.all(np.abs(xy[:, 1]) < min(0.4, 0.45 - 0.04 - r))


def test_disks_refuse_an_impossible_packing():
    with pytest.raises(RuntimeError):
        W.disks(50, 0.2, 0.1, 2.0, 10.0, seed=1, max_tries=20_000)


@pytest.mark.parametrize("k1,n", [(40.0, 1), (10.0, 1), (80.0, 3)])
def test_wood_angle_closed_form(k1, n):
    th = W.wood_angle(k1, 1.0, n)
    kappa_n = k1 * math.cos(th) + 2 * math.pi * n          # kappa_n = kappa + 2 pi n / d, d = 1
    assert math.isclose(kappa_n, k1, rel_tol=0, abs_tol=1e-12)
    assert k1 * k1 - kappa_n * kappa_n == pytest.approx(0.0, abs=1e-9)   # k_{1,n} = 0: grazing
    assert math.sin(th) < 0


def test_batched_angles_hold_the_wood_angle():
    th = W.batched_angles(40.0, 256)
    assert th.shape == (256,)
    phi = th + 0.5 * math.pi
    assert phi.min() >= -math.pi / 3 - 1e-15 and phi.max() <= math.pi / 3 + 1e-15
    assert np.any(th == W.wood_angle(40.0))
    assert np.all(np.sin(th) < 0)


def test_batched_geometries_uneven_sizes():
    geos = W.batched_geometries(n_geom=6, seed=4, m_lo=20, m_hi=200)
    Ms = [g["xy"].shape[0] for g in geos]
    assert all(20 <= m <= 200 for m in Ms) and len(set(Ms)) > 1
    for g in geos:
        r = g["radius"][0]
        assert 0.004 <= r <= 0.01
        assert np.sqrt(_min_image_dist2(g["xy"]).min()) >= 2.5 * r - 1e-15   # gap r/2
        assert np.all((g["kp"] >= 1.5 * 40.0) & (g["kp"] <= 2.5 * 40.0))


def test_sweep_points_ranges():
    s = W.sweep_points(1000, seed=5)
    assert s.shape == (1000, 2)
    assert np.all(np.abs(s[:, 0]) <= math.pi / 3) and np.all((s[:, 1] >= 35.0) & (s[:, 1] <= 45.0))
    np.testing.assert_array_equal(s, W.sweep_points(1000, seed=5))


@pytest.mark.parametrize("p", [3, 12])
def test_mlp_init_layout(p):
    w = W.mlp_init(p, seed=11)
    no = 2 * (2 * p + 1)
    assert w.dtype == np.float32
    assert w.size == 64 * 128 + 128 + 128 * 128 + 128 + 128 * no + no
    o = 64 * 128
    assert np.all(w[o:o + 128] == 0)                                  # b1
    o2 = o + 128 + 128 * 128
    assert np.all(w[o2:o2 + 128] == 0)                                # b2
    assert np.all(w[-no:] == 0)                                       # b3
    # weights N(0, 1/fan_in): the sample spread of W1 is close to 1/8
    assert abs(np.std(w[:o]) - 1.0 / 8.0) < 0.01
