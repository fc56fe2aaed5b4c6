"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong shift or index, a swapped operand) breaks at least one of them:
closed forms, published values, brute force on tiny inputs, an independent
second algorithm, and structural invariants.
"""
import math
import os
from itertools import combinations, permutations

import numpy as np
import pytest

import oracle
from paper_2604_05982_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------- hashing
def test_splitmix64_published_vector():
    state = 0
    for k, hexval in _read_golden("splitmix64_seed0.txt"):
        assert oracle.splitmix64(state) == int(hexval, 16), k
        state = (state + 0x9E3779B97F4A7C15) & (2 ** 64 - 1)


def test_input_stream_matches_published_vector():
    # the shared input generator follows the same published definition
    vals = inputs.splitmix64_stream(0, 0, 3)
    want = [int(h, 16) for _, h in _read_golden("splitmix64_seed0.txt")]
    assert [int(v) for v in vals] == want


# --------------------------------------------------------------------------- fib
def _fib_fast_doubling(n):
    # F(2k) = F(k) (2F(k+1) - F(k)), F(2k+1) = F(k)^2 + F(k+1)^2
    def fd(k):
        if k == 0:
            return 0, 1
        a, b = fd(k >> 1)
        c = a * (2 * b - a)
        d = a * a + b * b
        return (d, c + d) if k & 1 else (c, d)
    return fd(n)[0]


def test_fib_closed_form_and_task_count():
    for n in range(0, 27):
        v, t = oracle.fib(n)
        assert v == _fib_fast_doubling(n)
        # every call is one task: T(n) = 1 + T(n-1) + T(n-2), T(0)=T(1)=1 -> 2F(n+1) - 1
        assert t == 2 * _fib_fast_doubling(n + 1) - 1
    assert oracle.fib(30) == (832040, 2692537)


def test_fib_binet():
    phi = (1 + 5 ** 0.5) / 2
    for n in (10, 20, 30):
        assert oracle.fib(n)[0] == round(phi ** n / 5 ** 0.5)


def test_fib_cutoff_value_and_task_count_closed_form():
    # calls below the cutoff c >= 2 are leaf tasks: T(n) = 1 for n < c, else 1 + T(n-1) + T(n-2),
    # so T(n) + 1 follows the Fibonacci recurrence from T(c-2) + 1 = T(c-1) + 1 = 2:
    # T(n) = 2 F(n - c + 3) - 1 for n >= c - 2
    for c in range(2, 12):
        for n in range(max(0, c - 2), 28):
            v, t = oracle.fib_cutoff(n, c)
            assert v == _fib_fast_doubling(n)
            assert t == 2 * _fib_fast_doubling(n - c + 3) - 1, (n, c)
    # cutoff 0, 1 and 2 are the no-cutoff program
    for c in (0, 1, 2):
        assert oracle.fib_cutoff(25, c) == oracle.fib(25)


# --------------------------------------------------------------------------- n-queens
def _partial_placements_rows(n, rows):
    # brute force: valid placements of r queens in rows 0..r-1, for each r <= rows
    total = 0
    for r in range(min(rows, n) + 1):
        for cols in permutations(range(n), r):
            if all(abs(cols[i] - cols[j]) != j - i for i in range(r) for j in range(i + 1, r)):
                total += 1
    return total


def test_nqueens_cutoff_solutions_and_task_count():
    # the solutions do not depend on the cutoff; the tasks are the boards with at most
    # `depth` rows placed (brute-force count of partial placements)
    for n in range(1, 9):
        for depth in range(0, n + 2):
            s, t = oracle.nqueens_cutoff(n, depth)
            assert s == oracle.nqueens(n)[0]
            assert t == _partial_placements_rows(n, depth), (n, depth)
    assert oracle.nqueens_cutoff(11, 30) == oracle.nqueens(11)


def test_nqueens_published_counts():
    for n, sols in _read_golden("nqueens_solutions.txt"):
        n, sols = int(n), int(sols)
        assert oracle.nqueens(n)[0] == sols, n


def test_nqueens_permutation_brute_force():
    for n in range(1, 10):
        assert oracle.nqueens(n)[0] == oracle.nqueens_permutations(n)


def _partial_placements(n):
    # brute force over column tuples: count valid placements of r queens in rows 0..r-1
    total = 0
    for r in range(n + 1):
        for cols in permutations(range(n), r):
            if all(abs(cols[i] - cols[j]) != j - i for i in range(r) for j in range(i + 1, r)):
                total += 1
    return total


def test_nqueens_task_count_brute_force():
    for n in range(1, 8):
        assert oracle.nqueens(n)[1] == _partial_placements(n), n


def test_nqueens_two_algorithms_agree():
    for n in range(1, 12):
        assert oracle.nqueens(n, "bitmask") == oracle.nqueens(n, "array"), n


# --------------------------------------------------------------------------- hashed tree
def test_uts_recursion_equals_bfs():
    for seed, rc, m, thr in [(42, 2000, 5, oracle.UTS_THRESHOLD_Q0199), (1, 50, 3, 2 ** 62),
                             (7, 10, 2, 2 ** 63 - 2 ** 60), (3, 100, 1, 2 ** 64 - 2 ** 58)]:
        assert oracle.uts(seed, rc, m, thr) == oracle.uts(seed, rc, m, thr, algorithm="bfs")


def test_uts_special_cases():
    assert oracle.uts(42, 2000, 5, 0) == (2001, 2000)   # nobody below the root branches
    assert oracle.uts(42, 0, 5, 2 ** 63) == (1, 1)       # a lone root is a leaf
    assert oracle.uts(5, 1, 1, 0) == (2, 1)


def test_uts_counting_identity():
    # nodes = 1 + R + m * I and leaves = nodes - 1 - I, I = internal non-root nodes
    # all subcritical (m * q < 1), so every tree is finite
    for seed, rc, m, thr in [(42, 2000, 5, oracle.UTS_THRESHOLD_Q0199), (9, 300, 4, 2 ** 64 // 5),
                             (11, 64, 3, 2 ** 62)]:
        nodes, leaves = oracle.uts(seed, rc, m, thr)
        assert (nodes - 1 - rc) % m == 0
        internal = (nodes - 1 - rc) // m
        assert leaves == nodes - 1 - internal


def test_uts_branching_threshold_exact():
    assert oracle.UTS_THRESHOLD_Q0199 == 3670902070668200771
    assert oracle.UTS_THRESHOLD_Q0199 <= 0.199 * 2 ** 64 < oracle.UTS_THRESHOLD_Q0199 + 1 + 2 ** 12


def test_uts_branching_frequency():
    # a root with many children: the fraction of branching children estimates q
    nodes, leaves = oracle.uts(123, 200000, 1, 2 ** 62)   # q = 1/4, m = 1 chains
    # with m = 1, every non-root node except chain ends is internal: E[nodes-1] = R / (1 - q)
    assert abs((nodes - 1) / 200000 - 4 / 3) < 0.02


# --------------------------------------------------------------------------- sort
def test_bintree_task_counts_closed_form():
    # thread mode: every node of the full tree is a task; block mode with cutoff c:
    # the nodes of levels 0 .. D - c (a node c levels above the leaves is one task)
    for d in range(0, 11):
        assert oracle.bintree(d, 1)[1] == 2 ** (d + 1) - 1
        for c in (1, 3, 5):
            assert oracle.bintree(d, 1, cutoff=c)[1] == (2 ** (d - c + 1) - 1 if c < d else 1)


def test_bintree_recursion_equals_flat_leaf_enumeration():
    # the recursion's result is the sum over the leaf ids 2^D .. 2^(D+1)-1 of their
    # values (mod 2^64), whatever the cutoff
    for d, iters, k in [(0, 5, 1), (4, 3, 2), (7, 2, 4), (9, 1, 3)]:
        flat = sum(oracle.bintree_leaf(v, iters, k) for v in range(2 ** d, 2 ** (d + 1))) % 2 ** 64
        for c in (0, 2, 5):
            assert oracle.bintree(d, iters, k, cutoff=c)[0] == flat


def test_bintree_leaf_special_cases():
    # no iterations: every leaf is 0; the loop value is additive in the iteration range
    assert oracle.bintree(6, 0, 4)[0] == 0
    # K = 1 runs function 0 everywhere; a K = 4 leaf whose selected function is 0 has
    # the K = 1 value, and a leaf's value over n + 1 iterations adds one term to n
    sel = {}
    for v in range(64, 128):
        k4 = (oracle.splitmix64(v) >> 32) % 4
        sel[v] = k4
        if k4 == 0:
            assert oracle.bintree_leaf(v, 7, 4) == oracle.bintree_leaf(v, 7, 1)
    assert set(sel.values()) == {0, 1, 2, 3}
    # f0(0) = f1(0) = f3(0) = 0: leaf 0 with one iteration (input 0 << 32 = 0)
    assert oracle.bintree_leaf(0, 1, 1) == 0


def test_sort_is_sorted_permutation():
    keys = inputs.keys_u32(1 << 16, seed=1)
    out = oracle.sort_u32(keys)
    assert np.all(out[1:] >= out[:-1])
    ku, kc = np.unique(keys, return_counts=True)
    ou, oc = np.unique(out, return_counts=True)
    assert np.array_equal(ku, ou) and np.array_equal(kc, oc)
    edge = np.array([5, 5, 0, 2 ** 32 - 1, 7, 0], dtype=np.uint32)
    assert oracle.sort_u32(edge).tolist() == [0, 0, 5, 5, 7, 2 ** 32 - 1]


# --------------------------------------------------------------------------- integrate
def test_cilksort_sorts_and_counts_tasks():
    rng = np.random.default_rng(5)
    for n, sc, mc in [(0, 64, 256), (1, 64, 256), (63, 64, 256), (1000, 64, 256), (4096, 16, 32), (77777, 64, 256)]:
        keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
        if n > 10:
            keys[: n // 10] = keys[0]          # duplicates
        out, tasks = oracle.cilksort(keys, sc, mc)
        assert np.array_equal(out, np.sort(keys))
        if n == 0:
            assert tasks == 0
    # merges never split (merge cutoff >= n): the tasks are the sort recursion's 2L - 1
    # nodes (L leaves of <= sort_cutoff keys; n = 2^k * c splits into 2^k leaves) plus one
    # merge per inner node
    for k, c in [(0, 64), (3, 64), (6, 50)]:
        n = (2 ** k) * c
        _, tasks = oracle.cilksort(np.arange(n, dtype=np.uint32)[::-1].copy(), c, n)
        assert tasks == (2 ** (k + 1) - 1) + (2 ** k - 1)
    # merge cutoff 1: every merge task with more outputs places one key and forks two
    # smaller merges, so the merge tasks form a binary tree with one split task per key
    # placed: two leaves of one key (sort tasks 3) merge through 1 split + 2 leaf tasks
    for keys in ([3, 1], [1, 3], [2, 2]):
        out, tasks = oracle.cilksort(np.array(keys, dtype=np.uint32), 1, 1)
        assert list(out) == sorted(keys) and tasks == 3 + 3
    # every split task places one key and the leaves place the rest
    for n in (5, 64, 999):
        keys = rng.integers(0, 50, n, dtype=np.uint64).astype(np.uint32)
        out, _ = oracle.cilksort(keys, 1, 1)
        assert np.array_equal(out, np.sort(keys))


def test_integrate_close_to_closed_form():
    exact = 0.4 * math.atan(5.0)   # integral of 1/(1+25x^2) over [-1, 1]
    v, t = oracle.integrate_thread(-1.0, 1.0, 1e-10)
    assert abs(v - exact) < 1e-9 and t % 2 == 1
    vb, tb = oracle.integrate_block(-1.0, 1.0, 1e-10, 256)
    assert abs(vb - exact) < 1e-9 and tb % 2 == 1
    # [0, 1] is half of the symmetric integral
    v0, _ = oracle.integrate_thread(0.0, 1.0, 1e-10)
    assert abs(v0 - exact / 2) < 1e-9


def test_integrate_block_single_task_when_smooth():
    # a tiny interval is accepted at once: one task, and the value is the Richardson step
    vb, tb = oracle.integrate_block(0.0, 1e-3, 1e-6, 128)
    assert tb == 1
    assert abs(vb - math.atan(5e-3) / 5) < 1e-15


# --------------------------------------------------------------------------- k-clique
def _ek(sizes, k):
    # elementary symmetric polynomial e_k
    e = [1] + [0] * k
    for s in sizes:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * s
    return e[k]


def test_kclique_brute_force_random():
    for seed in range(4):
        n, edges = inputs.random_graph(18, 0.55, seed)
        for k in range(3, 7):
            want = oracle.kclique_brute(n, edges, k)
            assert oracle.kclique(n, edges, k, "degree") == want
            assert oracle.kclique(n, edges, k, "id") == want


def test_kclique_complete_graph():
    n = 14
    edges = np.array(list(combinations(range(n), 2)), dtype=np.int32)
    for k in range(3, 9):
        assert oracle.kclique(n, edges, k) == math.comb(n, k)


def test_kclique_multipartite():
    sizes = [3, 1, 4, 2, 5]
    part = np.repeat(np.arange(len(sizes)), sizes)
    n = len(part)
    edges = np.array([(i, j) for i, j in combinations(range(n), 2) if part[i] != part[j]], dtype=np.int32)
    for k in range(3, 6):
        assert oracle.kclique(n, edges, k) == _ek(sizes, k)


def test_kclique_pivoting_against_brute_force_and_closed_forms():
    # pivoting is a second, independent counting algorithm: brute force on small random
    # graphs, C(n, k) on complete graphs, e_k on complete multipartite graphs
    for seed in range(4):
        n, e = inputs.random_graph(22, 0.45, seed)
        for k in (3, 4, 5, 6):
            assert oracle.kclique_pivot(n, e, k)[0] == oracle.kclique_brute(n, e, k), (seed, k)
    n = 30
    e = np.array(list(combinations(range(n), 2)), dtype=np.int32)
    for k in (3, 7, 12):
        assert oracle.kclique_pivot(n, e, k)[0] == math.comb(n, k)
    sizes = [3, 1, 4, 2, 5]
    part = np.repeat(np.arange(len(sizes)), sizes)
    nn = len(part)
    edges = np.array([(i, j) for i, j in combinations(range(nn), 2) if part[i] != part[j]], dtype=np.int32)
    for k in range(3, 6):
        assert oracle.kclique_pivot(nn, edges, k)[0] == _ek(sizes, k)


def test_kclique_pivoting_equals_orientation_on_rmat():
    # the two algorithms agree on every k, whole graph and per DAG-edge range
    n, e = inputs.rmat_graph(10, 16, seed=7)
    m = len(e)
    for k in (3, 4, 5, 6, 7):
        assert oracle.kclique_pivot(n, e, k)[0] == oracle.kclique(n, e, k), k
    for lo, hi in [(0, 100), (m // 2, m // 2 + 57), (m - 30, m)]:
        assert oracle.kclique_pivot(n, e, 5, lo, hi)[0] == oracle.kclique_edge_range(n, e, 5, lo, hi)


def test_kclique_pivoting_all_sizes_matches_per_k():
    # one pass for every size equals the per-k pivot counts and the orientation counts
    n, e = inputs.rmat_graph(9, 16, seed=11)
    off, adj = oracle.orient(n, e)
    m = len(e)
    allk = oracle.kclique_pivot_all(off, adj, [(0, m)], 9)
    for k in range(3, 10):
        assert allk[k] == oracle.kclique_pivot(n, e, k)[0] == oracle.kclique(n, e, k), k
    # ranges add up
    parts = [oracle.kclique_pivot_all(off, adj, [(lo, min(m, lo + 700))], 6) for lo in range(0, m, 700)]
    assert [sum(p[k] for p in parts) for k in range(7)] == allk[:7]
    # complete graph
    kn = np.array(list(combinations(range(25), 2)), dtype=np.int32)
    o2, a2 = oracle.orient(25, kn)
    got = oracle.kclique_pivot_all(o2, a2, [(0, len(kn))], 12)
    assert got[3:] == [math.comb(25, k) for k in range(3, 13)]


def test_kclique_triangles_trace():
    n, edges = inputs.random_graph(120, 0.2, 11)
    A = np.zeros((n, n), dtype=np.int64)
    A[edges[:, 0], edges[:, 1]] = 1
    A[edges[:, 1], edges[:, 0]] = 1
    assert oracle.kclique(n, edges, 3) == int(np.trace(A @ A @ A)) // 6


def test_kclique_per_edge_sums_and_small_rmat():
    n, edges = inputs.rmat_graph(9, 16, seed=7)
    for k in (3, 4, 5):
        total, pe = oracle.kclique(n, edges, k, per_edge=True)
        assert int(pe.sum()) == total
        assert oracle.kclique(n, edges, k, "id") == total


def test_orientation_is_a_dag_with_sorted_lists():
    n, edges = inputs.rmat_graph(8, 8, seed=3)
    off, adj = oracle.orient(n, edges)
    deg = np.bincount(edges.ravel(), minlength=n)
    assert off[-1] == len(edges)
    for u in range(n):
        out = adj[off[u]:off[u + 1]]
        assert np.all(np.diff(out) > 0)
        for v in out:
            assert (deg[u], u) < (deg[v], v)


# --------------------------------------------------------------------------- generators
def test_rmat_generator_shape():
    n, edges = inputs.rmat_graph(10, 16, seed=7)
    assert n == 1024
    assert np.all(edges[:, 0] < edges[:, 1])
    key = edges[:, 0].astype(np.int64) * n + edges[:, 1]
    assert np.all(np.diff(key) > 0)          # sorted, no duplicates
    deg = np.bincount(edges.ravel(), minlength=n)
    assert deg[0] == deg.max()               # a = 0.57 skews mass to vertex 0


def test_keys_u32_low_bits():
    k = inputs.keys_u32(4, seed=0)
    want = [int(h, 16) & 0xFFFFFFFF for _, h in _read_golden("splitmix64_seed0.txt")]
    assert k[:3].tolist() == want


def test_kclique_edge_range_sums_per_edge_counts():
    n, edges = inputs.rmat_graph(9, 16, seed=5)
    total, pe = oracle.kclique(n, edges, 4, per_edge=True)
    m = len(edges)
    assert oracle.kclique_edge_range(n, edges, 4, 0, m) == total
    for lo, hi in [(0, 10), (37, 400), (m - 5, m)]:
        assert oracle.kclique_edge_range(n, edges, 4, lo, hi) == int(pe[lo:hi].sum())


def test_kclique_dag_ranges_on_a_preoriented_graph():
    # several ranges of an already oriented DAG sum the per-edge counts of those ranges
    n, edges = inputs.rmat_graph(9, 16, seed=5)
    off, adj = oracle.orient(n, edges)
    m = len(edges)
    for k in (3, 4, 5):
        total, pe = oracle.kclique(n, edges, k, per_edge=True)
        assert oracle.kclique_dag_ranges(off, adj, k, [(0, m)]) == total
        ranges = [(0, 10), (37, 400), (m - 5, m), (500, 500)]
        assert oracle.kclique_dag_ranges(off, adj, k, ranges) == sum(int(pe[lo:hi].sum()) for lo, hi in ranges)


# ---------------------------------------------------------------------------
# Laplace FMM (Sec. 6.4.1).  The plain definition is the direct sum
# phi_i = sum_{j != i} q_j / |x_i - x_j|; the pins below tie the stepwise
# oracle to it (exactly where the method is exact, by convergence where it
# approximates) and check the traversal's lists and the tree independently.

def test_taylor_coefficients_closed_forms_and_series():
    r = np.array([0.7, -0.4, 1.1])
    x, y, z = r
    R = np.linalg.norm(r)
    T = oracle.taylor(4, r)
    idx = {m: i for i, m in enumerate(oracle.multi_indices(4))}
    assert T[idx[(0, 0, 0)]] == pytest.approx(1 / R, rel=1e-15)
    assert T[idx[(1, 0, 0)]] == pytest.approx(-x / R**3, rel=1e-14)
    assert T[idx[(0, 0, 1)]] == pytest.approx(-z / R**3, rel=1e-14)
    assert T[idx[(2, 0, 0)]] == pytest.approx((3 * x * x - R * R) / (2 * R**5), rel=1e-13)
    assert T[idx[(1, 1, 0)]] == pytest.approx(3 * x * y / R**5, rel=1e-13)
    assert T[idx[(1, 1, 1)]] == pytest.approx(-15 * x * y * z / R**7, rel=1e-13)
    assert T[idx[(3, 0, 0)]] == pytest.approx(-(5 * x**3 - 3 * x * R * R) / (2 * R**7), rel=1e-13)
    # generating function: sum_n T_n(r) h^n = 1/|r + h| for |h| < |r|, every order
    p = 12
    T = oracle.taylor(p, r)
    h = np.array([0.05, 0.03, -0.04])
    s = sum(T[i] * h[0]**a * h[1]**b * h[2]**c for i, (a, b, c) in enumerate(oracle.multi_indices(p)))
    assert s == pytest.approx(1 / np.linalg.norm(r + h), rel=1e-13)


@pytest.mark.parametrize("dist", ["uniform", "plummer"])
def test_fmm_single_leaf_is_the_direct_sum(dist):
    pos, q = inputs.fmm_points(64, dist)
    phi, m2l, p2p, nc = oracle.fmm(pos, q, lists=True)
    assert nc == 1 and len(m2l) == 0 and p2p.tolist() == [[0, 0]]
    np.testing.assert_allclose(phi, oracle.direct(pos, q), rtol=1e-13, atol=0)


@pytest.mark.parametrize("dist", ["uniform", "plummer"])
def test_fmm_tiny_theta_is_the_direct_sum(dist):
    pos, q = inputs.fmm_points(1500, dist)
    phi, m2l, p2p, nc = oracle.fmm(pos, q, theta=1e-9, leaf_size=16, lists=True)
    assert nc > 50 and len(m2l) == 0
    d = oracle.direct(pos, q)
    assert np.abs(phi - d).max() <= 1e-12 * np.abs(d).max()


@pytest.mark.parametrize("dist", ["uniform", "plummer"])
def test_fmm_error_falls_with_expansion_order(dist):
    pos, q = inputs.fmm_points(4096, dist)
    d = oracle.direct(pos, q)
    errs = [np.linalg.norm(oracle.fmm(pos, q, p=p) - d) / np.linalg.norm(d) for p in (2, 4, 6, 8)]
    for lo, hi in zip(errs[1:], errs[:-1]):
        assert lo < hi / 4
    assert errs[-1] < 3e-6


@pytest.mark.parametrize("dist", ["uniform", "plummer"])
def test_fmm_lists_cover_every_ordered_pair_once(dist):
    n, theta = 700, 0.5
    pos, q = inputs.fmm_points(n, dist)
    _, m2l, p2p, nc = oracle.fmm(pos, q, p=2, theta=theta, leaf_size=16, lists=True)
    cells, order = oracle.fmm_tree(pos, leaf_size=16)
    assert len(cells) == nc
    side = (pos.max(axis=0) - pos.min(axis=0)).max()
    members = [order[int(c[1]):int(c[1] + c[2])] for c in cells]
    cover = np.zeros((n, n), dtype=np.int32)
    for a, b in m2l:
        A, B = cells[a], cells[b]
        hA, hB = side / 2.0 ** (A[0] + 1), side / 2.0 ** (B[0] + 1)
        dist_ab = np.linalg.norm(A[5:8] - B[5:8])
        assert (hA + hB) * math.sqrt(3.0) < theta * dist_ab * (1 + 1e-12)
        cover[np.ix_(members[a], members[b])] += 1
    for a, b in p2p:
        assert cells[a, 3] < 0 and cells[b, 3] < 0
        cover[np.ix_(members[a], members[b])] += 1
    assert (cover == 1).all()


def test_fmm_tree_invariants():
    pos, q = inputs.fmm_points(5000, "plummer")
    cells, order = oracle.fmm_tree(pos, leaf_size=64)
    assert sorted(order.tolist()) == list(range(5000))
    side = (pos.max(axis=0) - pos.min(axis=0)).max()
    lvl = cells[:, 0]
    assert (np.diff(lvl) >= 0).all()                       # breadth-first numbering
    for i, c in enumerate(cells):
        level, first, count, child, nchild = int(c[0]), int(c[1]), int(c[2]), int(c[3]), int(c[4])
        h = side / 2.0 ** (level + 1)
        pts = pos[order[first:first + count]]
        assert (np.abs(pts - c[5:8]) <= h * (1 + 1e-12)).all()
        if child < 0:
            assert count <= 64 or level == 21
        else:
            assert count > 64 and 1 <= nchild <= 8
            kids = cells[child:child + nchild]
            assert (kids[:, 0] == level + 1).all()
            assert kids[0, 1] == first and kids[:, 2].sum() == count
            assert (kids[1:, 1] == kids[:-1, 1] + kids[:-1, 2]).all()


def test_fmm_target_subset_matches_full_run():
    pos, q = inputs.fmm_points(3000, "uniform")
    full = oracle.fmm(pos, q)
    tg = np.array([0, 17, 2999, 1234, 640], dtype=np.int64)
    np.testing.assert_array_equal(oracle.fmm(pos, q, targets=tg), full[tg])
