"""Pins for the FP64 PageRank oracle (Eq. 1 / Algorithm 1 plus the dangling
reading). Each pin comes from outside the oracle: a closed form derived by hand
from Eq. 1, a dense linear solve (numpy.linalg.solve) of the fixed-point
equation, or an invariant of the iteration. Between them a dropped term (the
teleport (1-d)/n, the dangling share D/n, the 1/outdeg scaling), a wrong sign,
or a transposed adjacency (out- instead of in-neighbours) fails at least one.
"""
import itertools

import numpy as np
import pytest

import graphgen
import oracle

D = 0.85


def cycle(n):
    return graphgen.csr_from_edges(n, np.arange(n), (np.arange(n) + 1) % n)


def bidirectional_star(n):
    leaves = np.arange(1, n)
    return graphgen.csr_from_edges(n, np.r_[np.zeros(n - 1, int), leaves], np.r_[leaves, np.zeros(n - 1, int)])


def in_star(n):
    leaves = np.arange(1, n)
    return graphgen.csr_from_edges(n, leaves, np.zeros(n - 1, int))


@pytest.mark.parametrize("n", [1, 2, 7, 64])
@pytest.mark.parametrize("dangling", ["uniform", "leak"])
def test_cycle_uniform_fixed_point(n, dangling):
    # Every node has one in- and one out-neighbour: 1/n is a fixed point of Eq. 1,
    # reached exactly from the uniform start on every iteration.
    if n == 1:
        rp, col = np.array([0, 0], np.uint32), np.array([], np.uint32)
        if dangling == "leak":
            pytest.skip("a lone node is dangling")
    else:
        rp, col = cycle(n)
    out = oracle.pagerank(rp, col, D, iters=5, dangling=dangling, history=True)
    np.testing.assert_allclose(out["hist"], 1.0 / n, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [2, 5, 17, 100])
@pytest.mark.parametrize("d", [0.5, 0.85, 0.99])
def test_bidirectional_star_closed_form(n, d):
    # Centre c <-> n-1 leaves, no dangling node. From Eq. 1:
    #   x_c = (1-d)/n + d (n-1) x_l,  x_l = (1-d)/n + d x_c/(n-1)
    # => x_c = (1 + d(n-1)) / (n(1+d)).
    rp, col = bidirectional_star(n)
    iters = int(np.ceil(np.log(1e-16) / np.log(d))) + 20
    x = oracle.pagerank(rp, col, d, iters=iters)["x"]
    xc = (1 + d * (n - 1)) / (n * (1 + d))
    xl = (1 - d) / n + d * xc / (n - 1)
    np.testing.assert_allclose(x[0], xc, rtol=1e-12)
    np.testing.assert_allclose(x[1:], xl, rtol=1e-12)
    assert abs(x.sum() - 1) < 1e-12


@pytest.mark.parametrize("n", [2, 3, 10, 50])
def test_in_star_dangling_centre_uniform(n):
    # Leaves -> centre; the centre is dangling and its mass returns uniformly:
    #   x_l = 1/(n + d(n-1)),  x_c = (1 + d(n-1)) / (n + d(n-1)).
    rp, col = in_star(n)
    x = oracle.pagerank(rp, col, D, iters=300)["x"]
    den = n + D * (n - 1)
    np.testing.assert_allclose(x[1:], 1 / den, rtol=1e-12)
    np.testing.assert_allclose(x[0], (1 + D * (n - 1)) / den, rtol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 10, 50])
def test_in_star_dangling_centre_leak(n):
    # Eq. 1 taken literally: leaves get only the teleport term, the centre adds
    # d times the leaves' mass; the dangling centre's own mass is lost.
    rp, col = in_star(n)
    x = oracle.pagerank(rp, col, D, iters=300, dangling="leak")["x"]
    np.testing.assert_allclose(x[1:], (1 - D) / n, rtol=1e-12)
    np.testing.assert_allclose(x[0], (1 - D) / n * (1 + D * (n - 1)), rtol=1e-12)


def dense_solution(rp, col, d, dangling):
    """Solves (I - d M) x = ((1-d)/n) 1 with M = A^T D^+ (+ (1/n) 1 delta^T
    for uniform dangling), via numpy.linalg.solve."""
    n = rp.size - 1
    A = np.zeros((n, n))
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            A[u, col[e]] += 1.0
    outdeg = A.sum(axis=1)
    M = np.zeros((n, n))
    for u in range(n):
        if outdeg[u] > 0:
            M[:, u] = A[u, :] / outdeg[u]
        elif dangling == "uniform":
            M[:, u] = 1.0 / n
    return np.linalg.solve(np.eye(n) - d * M, np.full(n, (1 - d) / n))


def all_digraphs(n, self_loops):
    pairs = [(u, v) for u in range(n) for v in range(n) if self_loops or u != v]
    for mask in range(1 << len(pairs)):
        src = [pairs[i][0] for i in range(len(pairs)) if mask >> i & 1]
        dst = [pairs[i][1] for i in range(len(pairs)) if mask >> i & 1]
        yield graphgen.csr_from_edges(n, np.array(src, int), np.array(dst, int), drop_self_loops=False)


@pytest.mark.parametrize("n,self_loops", [(2, True), (3, True), (4, False)])
@pytest.mark.parametrize("dangling", ["uniform", "leak"])
def test_dense_solve_exhaustive(n, self_loops, dangling):
    worst = 0.0
    for rp, col in all_digraphs(n, self_loops):
        x = oracle.pagerank(rp, col, D, iters=200, dangling=dangling)["x"]
        worst = max(worst, np.abs(x - dense_solution(rp, col, D, dangling)).max())
    assert worst < 1e-12


@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("dangling", ["uniform", "leak"])
def test_dense_solve_random(seed, dangling):
    n = 5 + seed % 6
    rp, col = graphgen.random_graph(n, m_draws=2 * n + seed % 7, seed=seed, drop_self_loops=seed % 2 == 0)
    d = [0.5, 0.85, 0.9][seed % 3]
    x = oracle.pagerank(rp, col, d, iters=300, dangling=dangling)["x"]
    np.testing.assert_allclose(x, dense_solution(rp, col, d, dangling), rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_invariants_random_graph(seed):
    # Non-negativity, total mass 1 under uniform dangling, mass <= 1 under leak,
    # and the L1 step contracts by at least d per iteration (column-(sub)stochastic M).
    rp, col = graphgen.random_graph(300, m_draws=900, seed=100 + seed)
    x0 = graphgen.random_rank_vector(300, seed=7 + seed)
    for dangling in ("uniform", "leak"):
        out = oracle.pagerank(rp, col, D, iters=30, x0=x0, dangling=dangling, history=True)
        h = out["hist"]
        assert (h >= 0).all()
        if dangling == "uniform":
            np.testing.assert_allclose(h.sum(axis=1), 1.0, atol=1e-13)
        else:
            assert (h.sum(axis=1) <= 1 + 1e-13).all()
        r = out["resid"]
        np.testing.assert_allclose(r, np.abs(np.diff(h, axis=0)).sum(axis=1), rtol=1e-12)
        assert (r[1:] <= D * r[:-1] * (1 + 1e-9) + 1e-15).all()


def test_history_matches_restart():
    # x_i from one run equals x_1 of a run started at x_{i-1}: the iteration
    # carries no hidden state besides the vector.
    rp, col = graphgen.rmat(8, 8, seed=3)
    full = oracle.pagerank(rp, col, D, iters=6, history=True)["hist"]
    for i in range(1, 7):
        step = oracle.pagerank(rp, col, D, iters=1, x0=full[i - 1])["x"]
        np.testing.assert_allclose(step, full[i], rtol=1e-15, atol=0)


def test_transpose_matters():
    # A path 0 -> 1 -> 2 with the uniform start: after one step node 0 holds only
    # the teleport share plus dangling share, node 1 and 2 receive d * x(u)/1.
    rp, col = graphgen.csr_from_edges(3, np.array([0, 1]), np.array([1, 2]))
    x1 = oracle.pagerank(rp, col, D, iters=1)["x"]
    base = (1 - D) / 3 + D * (1 / 3) / 3  # node 2 is dangling with mass 1/3
    np.testing.assert_allclose(x1, [base, base + D / 3, base + D / 3], rtol=1e-15)


def test_pull_step_ranges_compose():
    # Steps over disjoint destination ranges assemble the full step.
    rp, col = graphgen.rmat(10, 16, seed=21)
    n = rp.size - 1
    x0 = graphgen.random_rank_vector(n, seed=22)
    full = oracle.pagerank(rp, col, D, iters=1, x0=x0)
    pull = oracle.Pull(rp, col)
    y = np.zeros(n)
    r = sum(pull.step(x0, y, D, v_begin=a, v_end=min(n, a + 100)) for a in range(0, n, 100))
    np.testing.assert_array_equal(y, full["x"])
    np.testing.assert_allclose(r, full["resid"][0], rtol=1e-12)
    assert pull.in_edges(0, n) == rp[-1]


@pytest.mark.parametrize("threads", [2, 3, 8])
@pytest.mark.parametrize("dangling", ["uniform", "leak"])
def test_threaded_oracle_matches_sequential(threads, dangling):
    # The threaded step computes every y[v] exactly as the sequential one
    # (same in-neighbour order); only the pieces' L1 sums are added in
    # another order. Ragged pieces: n is not a multiple of the thread count.
    rp, col = graphgen.rmat(11, 8, seed=4242)
    ref = oracle.pagerank(rp, col, D, iters=7, dangling=dangling, history=True)
    got = oracle.pagerank(rp, col, D, iters=7, dangling=dangling, history=True, threads=threads)
    np.testing.assert_array_equal(got["hist"], ref["hist"])
    np.testing.assert_allclose(got["resid"], ref["resid"], rtol=1e-13, atol=0)
    pull = oracle.Pull(rp, col)
    x = ref["hist"][3]
    y1, y2 = np.empty_like(x), np.empty_like(x)
    r1 = pull.step(x, y1, D, dangling)
    r2 = pull.step_all(x, y2, D, dangling, threads=threads)
    np.testing.assert_array_equal(y1, y2)
    assert abs(r1 - r2) <= 1e-13 * r1
    assert oracle.host_threads() >= 1
