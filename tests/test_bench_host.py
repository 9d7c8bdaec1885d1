"""Host-side arithmetic of bench.py (CPU)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_launch_count_of_a_solve():
    """A config-2 solve of 38 iterations, checked every 8, launches 40
    iterations of eight kernels (sweep, finalize, the zeroing of the skewed
    T_L partials, the finalisation tail, three Anderson kernels, the records'
    difference fields) plus the first guess and five start-of-solve kernels:
    326 kernels of the library."""
    import bench
    assert bench.launches_per_solve(38, 8) == 326
    assert bench.launches_per_solve(32, 8) == 6 + 8 * 32
    assert bench.launches_per_solve(1, 8) == 6 + 8 * 8


def test_sweep_blocks_of_the_warp_kernel():
    """Config 2: 1088 warp work items (groups padded to blocks of four of one
    quadrant) in blocks of 128 threads give the 272-block grid of the launch
    list; block kernels run one group per block."""
    import bench
    assert bench.sweep_blocks({"n_groups": 1088, "kernel": 2, "threads_per_block": 128}) == 272
    assert bench.sweep_blocks({"n_groups": 1081, "kernel": 2, "threads_per_block": 128}) == 271
    assert bench.sweep_blocks({"n_groups": 300, "kernel": 1, "threads_per_block": 256}) == 300
