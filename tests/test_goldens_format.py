"""The committed k-clique golden files are self-consistent (no GPU).

Their values come from the oracle alone (tests/golden/make_kclique_goldens.py);
these checks catch a truncated or hand-edited file: whole-graph files hold 64
ranges that partition the DAG edges and whose counts add up to the total;
sampled files hold 256 disjoint in-range ranges; the batch file holds one count
per graph with the stated scale and seed."""
import importlib.util
import os

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _mod():
    spec = importlib.util.spec_from_file_location("make_kclique_goldens", os.path.join(GOLDEN, "make_kclique_goldens.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_whole_graph_goldens_partition_and_sum():
    m = _mod()
    for k in (4, 5):
        g = m.load(os.path.join(GOLDEN, f"kclique_rmat20_k{k}.txt"))
        assert g["k"] == k and len(g["ranges"]) == m.N_RANGES
        assert [(lo, hi) for lo, hi, _ in g["ranges"]] == m.golden_ranges(g["m"])
        assert sum(c for _, _, c in g["ranges"]) == g["total"]
        assert all(c >= 0 for _, _, c in g["ranges"])
    # the files belong to the same graph, and hold the counts quoted in the documentation
    g4 = m.load(os.path.join(GOLDEN, "kclique_rmat20_k4.txt"))
    g5 = m.load(os.path.join(GOLDEN, "kclique_rmat20_k5.txt"))
    assert g4["m"] == g5["m"] == 15700209 and g4["n"] == g5["n"] == 1 << 20
    assert g4["total"] == 17080623729 and g5["total"] == 632099292765


def test_sampled_goldens_ranges():
    m = _mod()
    for k in (6, 7):
        g = m.load(os.path.join(GOLDEN, f"kclique_rmat20_k{k}_sampled.txt"))
        assert g["k"] == k and len(g["ranges"]) == 256
        assert [(lo, hi) for lo, hi, _ in g["ranges"]] == m.sampled_ranges(g["m"], 256, 4)
        assert all(c >= 0 for _, _, c in g["ranges"])


def test_batch_golden_graphs():
    m = _mod()
    g = m.load(os.path.join(GOLDEN, "kclique_batch64_k4.txt"))
    assert g["k"] == 4 and len(g["graphs"]) == 64
    for i, (gi, scale, seed, edges, count) in enumerate(g["graphs"]):
        assert gi == i and (scale, seed) == m.batch64_graph(i) and edges > 0 and count >= 0
