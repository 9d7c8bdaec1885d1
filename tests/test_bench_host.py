"""Host-side arithmetic of bench.py (CPU)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_launch_count_matches_the_launch_list():
    """The bench's own launch list (ncu, 5 solves of the config-2 workload at
    34 iterations each, check every 8) holds 1225 kernels of the library:
    40 launches each of the sweep, finalize, its tail and the three Anderson
    kernels, plus the first guess and four start-of-solve kernels, per solve."""
    import bench
    assert bench.launches_per_solve(34, 8) == 245
    assert 5 * bench.launches_per_solve(34, 8) == 1225
    assert bench.launches_per_solve(32, 8) == 5 + 6 * 32
    assert bench.launches_per_solve(1, 8) == 5 + 6 * 8


def test_sweep_blocks_of_the_warp_kernel():
    """Config 2: 1088 warp work items (groups padded to blocks of four of one
    quadrant) in blocks of 128 threads give the 272-block grid of the launch
    list; block kernels run one group per block."""
    import bench
    assert bench.sweep_blocks({"n_groups": 1088, "kernel": 2, "threads_per_block": 128}) == 272
    assert bench.sweep_blocks({"n_groups": 1081, "kernel": 2, "threads_per_block": 128}) == 271
    assert bench.sweep_blocks({"n_groups": 300, "kernel": 1, "threads_per_block": 256}) == 300
