"""The oracle's input encodings of Sec. 4 "Input Encoding" (CPU): the multiresolution
hash grid (8 levels x 2 features, resolution 16 doubling per level, 2^18 entries per
level), one-blob encodings, StatNet's 32 inputs and the 32-input MLP.  Pinned by what
holds whatever the implementation: trilinear interpolation reproduces linear functions
and sums weights to one, a grid vertex reads its own entry, the encoding is linear in the
table so its backward pass is its adjoint, the one-blob kernel peaks at the value's bin,
and the MLP's gradients match central differences."""
import numpy as np
import pytest

import oracle

T = 1 << 18
LEVELS = 8


def _level_table(level, fn0, fn1):
    """A table whose level `level` holds fn0 / fn1 of each dense vertex, other levels 0."""
    N = 16 << level
    n1 = N + 1
    assert n1 ** 3 <= T
    tab = np.zeros((LEVELS, T, 2))
    v = np.arange(n1 ** 3)
    x, y, z = v % n1, (v // n1) % n1, v // (n1 * n1)
    tab[level, v, 0] = fn0(x, y, z)
    tab[level, v, 1] = fn1(x, y, z)
    return tab.ravel()


@pytest.mark.parametrize("level", [0, 1])
def test_dense_levels_reproduce_linear_functions(level):
    N = 16 << level
    f0 = lambda x, y, z: 0.5 + 0.25 * x - 0.125 * y + 0.0625 * z
    f1 = lambda x, y, z: -1.0 + 0.01 * x + 0.02 * y + 0.03 * z
    tab = _level_table(level, f0, f1)
    rng = np.random.default_rng(level)
    p = np.vstack([rng.random((64, 3)), [[0, 0, 0], [1, 1, 1], [1, 0, 0.5]]])
    out = oracle.grid_encode(tab, p)
    s = p * N
    np.testing.assert_allclose(out[:, 2 * level], f0(*s.T), rtol=0, atol=1e-12)
    np.testing.assert_allclose(out[:, 2 * level + 1], f1(*s.T), rtol=0, atol=1e-12)
    others = [c for c in range(16) if c // 2 != level]
    assert np.all(out[:, others] == 0)


def test_weights_sum_to_one():
    out = oracle.grid_encode(np.ones(oracle.grid_param_count()),
                             np.random.default_rng(1).random((50, 3)))
    np.testing.assert_allclose(out, 1.0, rtol=0, atol=1e-12)


def test_vertex_reads_its_entry_and_hash():
    """At a grid vertex the feature is that vertex's entry: dense levels by the linear
    index, finer levels by the spatial hash (1, 2654435761, 805459861) mod 2^18."""
    tab = np.random.default_rng(2).normal(size=oracle.grid_param_count())
    tab3 = tab.reshape(LEVELS, T, 2)
    rng = np.random.default_rng(3)
    for level in range(LEVELS):
        N = 16 << level
        for _ in range(5):
            v = rng.integers(0, N + 1, 3)
            if (N + 1) ** 3 <= T:
                idx = v[0] + (N + 1) * (v[1] + (N + 1) * v[2])
            else:
                M = (1 << 32) - 1  # 32-bit unsigned products
                h = (int(v[0]) * 1 & M) ^ (int(v[1]) * 2654435761 & M) ^ (int(v[2]) * 805459861 & M)
                idx = h & (T - 1)
            assert oracle.grid_index(level, *map(int, v)) == idx
            out = oracle.grid_encode(tab, v / N)[0]
            np.testing.assert_allclose(out[2 * level:2 * level + 2], tab3[level, idx], atol=1e-12)


def test_continuous_across_cell_faces():
    tab = np.random.default_rng(4).normal(size=oracle.grid_param_count())
    p = np.array([5.0 / 16.0, 0.3, 0.7])
    a = oracle.grid_encode(tab, p - [1e-12, 0, 0])
    b = oracle.grid_encode(tab, p + [1e-12, 0, 0])
    np.testing.assert_allclose(a, b, atol=1e-7)


def test_backward_is_the_adjoint_of_the_encoding():
    """The encoding is linear in the table: <dout, encode(dT)> = <backward(dout), dT>."""
    rng = np.random.default_rng(5)
    p = rng.random((6, 3))
    dout = rng.normal(size=(6, 16))
    G = oracle.grid_backward(p, dout)
    for _ in range(3):
        dT = rng.normal(size=oracle.grid_param_count())
        lhs = float(np.sum(dout * oracle.grid_encode(dT, p)))
        assert abs(lhs - float(G @ dT)) <= 1e-9 * max(1.0, abs(lhs))
    # only the corners of the points' cells receive gradient
    assert np.count_nonzero(G) <= 6 * LEVELS * 8 * 2


def test_one_blob():
    for k in (4, 8):
        for i in range(k):
            out = oracle.one_blob((i + 0.5) / k, k)
            assert out[i] == 1.0 and np.argmax(out) == i
            if 0 < i < k - 1:
                assert abs(out[i - 1] - np.exp(-0.5)) < 1e-15 and out[i - 1] == out[i + 1]
    out = oracle.one_blob(0.3, 4)  # between bins 0 and 1: kernel exp(-((c - v) k)^2 / 2)
    np.testing.assert_allclose(out, np.exp(-0.5 * ((np.arange(4) + 0.5) / 4 - 0.3) ** 2 * 16),
                               rtol=1e-15)


def test_statnet_grid_inputs_layout():
    tab = np.random.default_rng(6).normal(size=oracle.grid_param_count())
    p = np.array([0.2, 0.6, 0.9])
    x = oracle.statnet_grid_inputs(tab, p, [0.0, 0.0, 1.0], 0.0)
    np.testing.assert_allclose(x[:16], oracle.grid_encode(tab, p)[0], atol=1e-15)
    np.testing.assert_allclose(x[16:20], oracle.one_blob(0.0, 4), atol=1e-15)  # theta = 0
    np.testing.assert_allclose(x[20:24], oracle.one_blob(0.5, 4), atol=1e-15)  # phi = 0
    np.testing.assert_allclose(x[24:32], oracle.one_blob(0.0, 8), atol=1e-15)  # alpha = 0
    x = oracle.statnet_grid_inputs(tab, p, [0.0, -1.0, 0.0], 1.0)  # theta = pi/2, phi = -pi/2
    np.testing.assert_allclose(x[16:20], oracle.one_blob(0.5, 4), atol=1e-15)
    np.testing.assert_allclose(x[20:24], oracle.one_blob(0.25, 4), atol=1e-15)
    np.testing.assert_allclose(x[24:32], oracle.one_blob(1 - np.exp(-1.0), 8), atol=1e-15)


def test_mlp32_gradients_match_central_differences():
    rng = np.random.default_rng(7)
    n_in, n_out = 32, 6
    P = rng.normal(size=oracle.mlpk_param_count(n_in, n_out)) * 0.3
    x = rng.normal(size=n_in)
    dout = rng.normal(size=n_out)
    G, dx = oracle.mlpk_backward(P, n_in, n_out, x, dout)
    f = lambda P_, x_: float(dout @ oracle.mlpk_forward(P_, n_in, n_out, x_))
    h = 1e-6
    for i in rng.choice(P.size, 40, replace=False):
        e = np.zeros_like(P)
        e[i] = h
        fd = (f(P + e, x) - f(P - e, x)) / (2 * h)
        assert abs(fd - G[i]) <= 1e-6 * max(1.0, abs(fd))
    for k in range(n_in):
        e = np.zeros(n_in)
        e[k] = h
        fd = (f(P, x + e) - f(P, x - e)) / (2 * h)
        assert abs(fd - dx[k]) <= 1e-6 * max(1.0, abs(fd))
    # 16 inputs: the same network as the RRSNet / StatNet one of the other tests
    P16 = rng.normal(size=oracle.mlpk_param_count(16, n_out))
    x16 = rng.normal(size=16)
    np.testing.assert_allclose(oracle.mlpk_forward(P16, 16, n_out, x16),
                               oracle.mlpn_forward(P16, n_out, x16), rtol=1e-15)
