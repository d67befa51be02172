"""Host logic of the benchmark: the count of (pixel, neighbour) pairs of a
dense sequence with clipped windows against brute force, the second-order
per-unit flop constants against their itemised definitions, the argument
checks that run before any GPU work, and the timed-frames label."""
import itertools

import pytest


def test_window_pairs_brute_force():
    import bench
    for W, H, F, r, T in ((7, 5, 4, 2, 3), (3, 9, 2, 3, 1), (1, 1, 5, 1, 2), (12, 6, 3, 3, 5)):
        n = 0
        for f, y, x in itertools.product(range(F), range(H), range(W)):
            for tau in range(max(0, f - T + 1), f + 1):
                for qy, qx in itertools.product(range(y - r, y + r + 1), range(x - r, x + r + 1)):
                    n += 0 <= qx < W and 0 <= qy < H
        assert bench._window_pairs(W, H, F, r, T) == n


def test_second_order_flop_constants():
    import bench
    n_aug = 56                                          # 55 unknowns + the log brightness
    per_neighbour = (14 + 18 + 1) + (45 + 56) + 2 * n_aug * (n_aug + 1) // 2
    assert bench.FLOP_PER_NEIGHBOUR_2 == per_neighbour
    trailing = sum(m * (m + 1) for m in range(1, 56))   # 2 flop x m(m+1)/2 entries per step
    solve = 2 * 54 + 2 * n_aug * (n_aug + 1) // 2 + 55 + trailing + sum(range(1, 56)) + 55 + 2
    assert bench.FLOP_PER_SOLVE_2 == solve
    assert trailing == 2 * 55 * 56 * 57 // 6


@pytest.mark.parametrize("argv", [["--form", "batching", "--batch-sequences", "0"],
                                  ["--form", "batching", "--batch-sequences", "49"],
                                  ["--warmup", "2"]])
def test_bench_rejects_bad_arguments_before_any_gpu_work(argv, monkeypatch, capsys):
    import sys
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    with pytest.raises(SystemExit) as e:
        bench.main()
    assert e.value.code == 2
    assert "error" in capsys.readouterr().err


def test_frames_timed_label():
    import bench
    assert bench._frames_timed(3, 20, 240) == "3-22"
    assert bench._frames_timed(5, 20, 240) == "5-24"
    assert bench._frames_timed(3, 237, 240) == "3-239"
    assert bench._frames_timed(3, 240, 240).startswith("3-239, then 0-2 with a reset")
