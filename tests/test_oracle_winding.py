"""Pins of the oracle's winding tags (Sec. 4.2 hook; rule stated in
oracle/winding.py): straight strings along each axis, orientation reversal,
a circular loop with an exactly countable number of pierced faces, and brute
force against wrapped atan2 phase sums."""
import math

import numpy as np
import pytest

from oracle import winding
from paper_2404_02950_gb300 import inputs


def _grid(n):
    ax = np.arange(n, dtype=np.float64)
    return np.meshgrid(ax, ax, ax, indexing="ij")   # Z, Y, X


@pytest.mark.parametrize("axis", ["x", "y", "z"])
@pytest.mark.parametrize("sign", [1, -1])
@pytest.mark.parametrize("profile", ["linear", "tanh"])
def test_straight_string_pierces_one_plaquette_per_layer(axis, sign, profile):
    n = 9
    Z, Y, X = _grid(n)
    c = {"x": 3.3, "y": 4.6, "z": 2.7}
    # (u, v) around each string axis, counter-clockwise about +axis
    uv = {"z": (X - c["x"], Y - c["y"]), "x": (Y - c["y"], Z - c["z"]),
          "y": (Z - c["z"], X - c["x"])}[axis]
    du, dv = uv
    r = np.hypot(du, dv)
    amp = r if profile == "linear" else np.tanh(0.7 * r) / np.maximum(r, 1e-300) * r
    th = np.arctan2(sign * dv, du)
    psi1, psi2 = amp * np.cos(th), amp * np.sin(th)
    W = winding.plaquette_winding(psi1, psi2, periodic=False)
    for w in "xyz":
        if w != axis:
            assert not W[w].any(), (axis, w)
    Wa = W[axis]
    nz_idx = np.argwhere(Wa != 0)
    assert np.all(Wa[Wa != 0] == sign)
    # exactly one pierced plaquette per layer along the string, at the
    # lower corner (floor of the off-lattice crossing point)
    along = {"x": 2, "y": 1, "z": 0}[axis]
    assert len(nz_idx) == n - 1
    assert sorted(nz_idx[:, along].tolist()) == list(range(n - 1))
    exp = {"z": (math.floor(c["y"]), math.floor(c["x"])),
           "x": (math.floor(c["z"]), math.floor(c["y"])),
           "y": (math.floor(c["z"]), math.floor(c["x"]))}[axis]
    other = [a for a in (0, 1, 2) if a != along]
    for row in nz_idx:
        assert tuple(row[other]) == exp


def test_circular_loop_pierced_face_count():
    n, R = 40, 11.0
    p1, p2, _, _ = inputs.string_loop(n, R, 1.0, 0.5)
    cx = n / 2.0 - 0.5 + 0.25
    cy = n / 2.0 - 0.5 + 0.125
    W = winding.plaquette_winding(p1, p2, periodic=False)
    assert not W["z"].any()
    assert np.all(np.abs(W["x"]) <= 1) and np.all(np.abs(W["y"]) <= 1)
    # the loop lies between two z-layers and crosses every lattice line
    # x = i with |i - cx| < R twice (x-normal faces), same for y
    exp_x = 2 * sum(1 for i in range(n) if abs(i - cx) < R)
    exp_y = 2 * sum(1 for j in range(n) if abs(j - cy) < R)
    assert np.count_nonzero(W["x"]) == exp_x
    assert np.count_nonzero(W["y"]) == exp_y


def _wrap(d):
    return (d + np.pi) % (2 * np.pi) - np.pi


def test_bruteforce_atan2_on_8cube():
    n = 8
    rng = np.random.default_rng(11)
    base = rng.standard_normal((2, 3, 3, 3))
    # smooth random field (few modes) so most plaquettes are away from ties
    Z, Y, X = _grid(n)
    f = [np.zeros((n, n, n)) for _ in range(2)]
    for c in range(2):
        for a in range(3):
            for b in range(3):
                for d in range(3):
                    f[c] += base[c, a, b, d] * np.cos(2 * np.pi * (a * X + b * Y + d * Z) / n + a - b)
    psi1, psi2 = f
    W = winding.plaquette_winding(psi1, psi2, periodic=True)
    th = np.arctan2(psi2, psi1)
    orient = {"z": ((0, 0, 1), (0, 1, 0)), "x": ((0, 1, 0), (1, 0, 0)), "y": ((1, 0, 0), (0, 0, 1))}
    checked = 0
    for w, (eu, ev) in orient.items():
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    p0 = (k, j, i)
                    p1 = tuple((p0[q] + eu[q]) % n for q in range(3))
                    p2 = tuple((p1[q] + ev[q]) % n for q in range(3))
                    p3 = tuple((p0[q] + ev[q]) % n for q in range(3))
                    cyc = [p0, p1, p2, p3, p0]
                    ds = [_wrap(th[cyc[e + 1]] - th[cyc[e]]) for e in range(4)]
                    if max(abs(x) for x in ds) > np.pi - 1e-6:
                        continue
                    wb = int(round(sum(ds) / (2 * np.pi)))
                    assert W[w][k, j, i] == wb, (w, k, j, i)
                    checked += 1
    assert checked > 0.9 * 3 * n ** 3
    assert sum(np.count_nonzero(W[w]) for w in W) > 0


def test_cell_tags_bruteforce_and_padded_agree():
    n = 8
    rng = np.random.default_rng(3)
    psi1, psi2 = rng.standard_normal((2, n, n, n))
    W = winding.plaquette_winding(psi1, psi2, periodic=True)
    orient = {"z": ((0, 0, 1), (0, 1, 0)), "x": ((0, 1, 0), (1, 0, 0)), "y": ((1, 0, 0), (0, 0, 1))}
    ref = np.zeros((n, n, n), dtype=np.uint8)
    for w, (eu, ev) in orient.items():
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    if W[w][k, j, i] == 0:
                        continue
                    for a in (0, 1):
                        for b in (0, 1):
                            q = tuple((np.array((k, j, i)) + a * np.array(eu) + b * np.array(ev)) % n)
                            ref[q] = 1
    assert np.array_equal(winding.cell_tags_periodic(psi1, psi2), ref)
    for g in (1, 2, 3):
        t = winding.cell_tags_padded(np.pad(psi1, g, mode="wrap"), np.pad(psi2, g, mode="wrap"), g)
        assert np.array_equal(t, ref)


def test_ties_and_axis_points():
    # X == 0 with opposite half planes: antipodal edge counts 0
    assert winding.edge_delta(1.0, 0.0, -1.0, -0.0) == 0
    # Im == 0 counts as upper half plane
    assert winding.edge_delta(-1.0, 0.0, -1.0, -1e-3) == 1     # crosses -x axis ccw
    assert winding.edge_delta(-1.0, -1e-3, -1.0, 0.0) == -1    # back, cw
    assert winding.edge_delta(1.0, 0.0, 1.0, -1e-3) == 0       # crosses +x axis
