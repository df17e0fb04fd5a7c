"""The paper workload's input generator against the model example it stands for (Sec. 6): geometry and
sources from the committed fixture, the model solution at hand-evaluated points."""

import json
import math
import os

import numpy as np

from paper_1703_01216_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_model_example.json")


def test_paper_workload_geometry_and_sources_follow_the_fixture():
    g = json.load(open(GOLD))
    w = I.paper_workload(64, 51, 51)
    lo, hi = g["R"]["x"]
    assert w.x0 == lo and abs(w.x0 + w.n * w.h - hi) < 1e-12
    dz = (g["R"]["z"][1] - g["R"]["z"][0]) / 51
    assert abs(w.zr[0] - (g["R"]["z"][0] + dz / 2)) < 1e-12 and abs(w.zr[-1] - (g["R"]["z"][1] - dz / 2)) < 1e-12
    assert abs(w.zy[0] - (g["Y"]["z"][0] + dz / 2)) < 1e-12 and abs(w.zy[-1] - (g["Y"]["z"][1] - dz / 2)) < 1e-12
    assert np.allclose(w.nu, dz) and w.Mp == g["M_prime"] and w.M == g["M"]
    r = g["source_offset_r"]
    want = sorted((cx * r, cy * r, z0) for z0 in g["source_planes_z0"] for cx, cy in g["source_cross_xy"])
    got = sorted(tuple(p) for p in w.sources[0])
    assert w.Q == 1 and np.allclose(np.array(got), np.array(want))


def test_model_solution_at_hand_evaluated_points():
    # a voxel-centred grid (h = 1, 21 points from -10) whose centres include x, y in {0, -4, 4, 5}
    n, h, x0 = 21, 1.0, -10.5
    zr = np.array([1.5, 1.3, 1.7])
    xi = I.paper_model_xi(n, x0, h, zr)
    idx = {v: int(v - x0 - 0.5) for v in (0.0, -4.0, 4.0, 5.0)}

    def model(x, y, z):
        a1 = (1 - 4 * (z - 1.5) ** 2) ** 2
        a2 = 0.4 * max(1 - (z - 1.3) ** 2, 0.0)
        a3 = 0.2 * max(1 - (z - 1.7) ** 2, 0.0) ** 2
        return (a1 * math.exp(-x * x - 2 * y * y) + a2 * math.exp(-3 * (x + 4) ** 2 - (y - 5) ** 2 + (x + 4) * (y - 5))
                + a3 * math.exp(-0.9 * ((x - 4) ** 2 + (y + 4) ** 2 + (x - 4) * (y + 4))))

    # the three bumps' centres (x, y) = (0, 0), (-4, 5), (4, -4) at depths 1.5, 1.3, 1.7
    for j, z in enumerate(zr):
        for (x, y) in ((0.0, 0.0), (-4.0, 5.0), (4.0, -4.0)):
            assert abs(xi[j, idx[y], idx[x]] - model(x, y, z)) <= 1e-14
    assert abs(xi[0, idx[0.0], idx[0.0]] - 1.0) < 1e-6           # a1 = 1 at z = 1.5, the others ~0
    assert abs(xi[1, idx[5.0], idx[-4.0]] - 0.4) < 1e-3           # a2 = 0.4 at z = 1.3 (a1 tiny there)
    assert abs(xi[2, idx[-4.0], idx[4.0]] - 0.2) < 1e-3           # a3 = 0.2 at z = 1.7


def test_synthetic_geometry_follows_the_stated_readings():
    """The synthetic workloads' geometry (readings 3, 4, 8): voxel-centred depths of R = [0.5, 1] with
    midpoint weights, one observation plane z = 0 disjoint from R, and source q the scaled cross
    (0, 0), (+-0.8, 0), (0, +-0.8) on the plane z = -0.1 (q + 1)."""
    w = I.config_workload(3)
    assert (w.n, w.Mp, w.Q, w.M, w.alphas.size) == (256, 64, 8, 1, 64)
    dz = 0.5 / 64
    assert np.allclose(w.zr, 0.5 + (np.arange(64) + 0.5) * dz) and np.allclose(w.nu, dz)
    assert np.array_equal(w.zy, [0.0]) and np.all(w.zr > 0)
    assert w.x0 == -1.0 and abs(w.x0 + w.n * w.h - 1.0) < 1e-15
    S = I.cross_sources(8)
    cross = {(0.0, 0.0), (-0.8, 0.0), (0.8, 0.0), (0.0, -0.8), (0.0, 0.8)}
    for q in range(8):
        assert {tuple(np.round(p[:2], 12)) for p in S[q]} == cross
        assert np.allclose(S[q, :, 2], -0.1 * (q + 1))
    assert np.allclose(np.log10(w.alphas), np.linspace(-8, -1, 64))
    # the phantom is the negative contrast and the data noise is unit-free (scaled by the level later)
    assert w.noise.shape == (8, 1, 256, 256) and w.noise_level == 0.01
