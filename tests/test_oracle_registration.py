"""Pins of the oracle's registration pieces (Sec. II-A labels as displacements, Sec. IV-B
priors, Eq. U_lin_comb with no seeds): the displacement grid, the patch dissimilarity against a
brute-force loop, identical images and an integer shift (the true displacement takes the
largest prior wherever its patch is inside the volume), rows of P summing to 1, and the fast
solve equal to the exact solve of Eq. (rw_eq) at m = N."""
import numpy as np

import synth
from oracle import eig, exact, graph, registration


def test_displacement_grid():
    d = registration.displacement_labels()
    assert d.shape == (27, 3)
    assert len({tuple(v) for v in d}) == 27
    np.testing.assert_array_equal(d[0], [-1, -1, -1])
    np.testing.assert_array_equal(d[1], [0, -1, -1])    # x fastest
    np.testing.assert_array_equal(d[13], [0, 0, 0])


def test_patch_sad_brute_force():
    dims = (5, 4, 3)
    rng = np.random.default_rng(1)
    F = rng.random(60)
    M = rng.random(60)
    d = registration.displacement_labels()[[0, 13, 22]]
    got = registration.patch_sad(F, M, dims, d, half=1)
    X, Y, Z = dims

    def at(a, x, y, z):
        x, y, z = min(max(x, 0), X - 1), min(max(y, 0), Y - 1), min(max(z, 0), Z - 1)
        return a[x + X * (y + Y * z)]
    for k, (dx, dy, dz) in enumerate(d):
        for z in range(Z):
            for y in range(Y):
                for x in range(X):
                    s = 0.0
                    for oz in (-1, 0, 1):
                        for oy in (-1, 0, 1):
                            for ox in (-1, 0, 1):
                                s += abs(at(F, x + ox, y + oy, z + oz)
                                         - at(M, x + ox + dx, y + oy + dy, z + oz + dz))
                    assert abs(got[x + X * (y + Y * z), k] - s) < 1e-12


def test_identical_images_and_integer_shift():
    dims = (9, 8, 7)
    F = synth.smooth_random_image(dims, seed=4, smooth=1.0, sigma=0.1)
    disp = registration.displacement_labels()
    P = registration.registration_priors(F, F, dims, disp, half=1)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-12)
    assert np.all(np.argmax(P, axis=1) == 13)
    # moving = fixed moved by d* = (1, 0, -1): M(y + d*) = F(y)
    ds = np.array([1, 0, -1])
    Fg = F.reshape(dims[::-1])
    Mg = np.empty_like(Fg)
    for z in range(dims[2]):
        for y in range(dims[1]):
            for x in range(dims[0]):
                sx, sy, sz = x - ds[0], y - ds[1], z - ds[2]
                sx, sy, sz = (min(max(sx, 0), dims[0] - 1), min(max(sy, 0), dims[1] - 1),
                              min(max(sz, 0), dims[2] - 1))
                Mg[z, y, x] = Fg[sz, sy, sx]
    P = registration.registration_priors(F, Mg.ravel(), dims, disp, half=1)
    kstar = int(np.nonzero((disp == ds).all(axis=1))[0][0])
    X, Y, Z = dims
    inner = [x + X * (y + Y * z) for z in range(2, Z - 2) for y in range(2, Y - 2)
             for x in range(2, X - 2)]
    assert np.all(np.argmax(P[inner], axis=1) == kstar)


def test_unseeded_fast_solve_is_exact_at_full_rank():
    dims = (6, 5, 4)
    F = synth.smooth_random_image(dims, seed=2, smooth=1.0, sigma=0.05)
    M = synth.smooth_random_image(dims, seed=3, smooth=1.0, sigma=0.05)
    g = graph.build_graph(F, dims, 50.0)
    disp = registration.displacement_labels()
    P = registration.registration_priors(F, M, dims, disp, half=1)
    lam, Q = eig.smallest_eigpairs(g.Lhat, g.N)
    r = registration.registration_solve(g, Q, lam, P, gamma=1.0, m=g.N, refine_steps=0)
    none = np.zeros(0, np.int64)
    Ue = exact.exact_rw(g, none, none, 27, P, 1.0)
    assert np.abs(r["U"] - Ue).max() < 1e-10
    np.testing.assert_allclose(Ue.sum(axis=1), 1.0, atol=1e-10)
    field = registration.expected_displacement(np.eye(27)[[13, 0]], disp)
    np.testing.assert_array_equal(field, [[0, 0, 0], [-1, -1, -1]])


def test_patch_sad_on_a_voxel_subset_equals_the_full_map():
    dims = (7, 6, 5)
    rng = np.random.default_rng(3)
    F, M = rng.random(210), rng.random(210)
    disp = registration.displacement_labels()
    full = registration.registration_priors(F, M, dims, disp, half=2)
    vox = np.array([0, 17, 104, 209])
    np.testing.assert_array_equal(registration.registration_priors(F, M, dims, disp, half=2,
                                                                   voxels=vox), full[vox])
