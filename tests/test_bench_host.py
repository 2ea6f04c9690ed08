"""Host logic of bench.py: the count of our kernel launches per EM iteration
that the bench line reports (gpu_launches), against counts written out by
hand from the structure of the fit graph."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_launch_count_nested_loop():
    b = _bench()
    # tensor-core loop, replacement every 50: 53 CG iterations run as a
    # segment of 50 (25 passes of two iterations) and one of 3 (2 passes,
    # the second copy of the last pass launched and returning at once);
    # 4 launches per iteration copy, 6 per replacement block (launched after
    # each inner segment, twice), cg_init and the M-step
    assert b.launches_per_em(53, 50, 4, 6, nested=True) == 1 + 27 * 2 * 4 + 2 * 6 + 1
    # a solve that ends exactly at a replacement (decided by its stop test):
    # no second segment and no second replacement block
    assert b.launches_per_em(50, 50, 4, 6, nested=True) == 1 + 25 * 2 * 4 + 1 * 6 + 1
    # B = 0: done at cg_init, the loops never run
    assert b.launches_per_em(0, 50, 4, 6, nested=True) == 2
    # odd segment: 37 iterations are 19 passes
    assert b.launches_per_em(37, 50, 4, 6, nested=True) == 1 + 19 * 2 * 4 + 1 * 6 + 1


def test_launch_count_single_loop():
    b = _bench()
    # CUDA-core loop with the replacement behind an IF node: one iteration
    # per pass, one replacement at iteration 50
    assert b.launches_per_em(53, 50, 6, 5) == 1 + 53 * 6 + 1 * 5 + 1
    assert b.launches_per_em(20, 0, 6, 5) == 1 + 20 * 6 + 1
