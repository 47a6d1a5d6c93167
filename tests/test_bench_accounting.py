"""Host-side accounting of bench.py's roofline line: the algorithmic bytes
and flops per FP64 BP3 apply of each order's default body, and the DRAM
traffic ratios of the committed captures."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import fem_inputs  # noqa: E402


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def packed_entries(P3):
    """(a, b) pairs of the packed upper triangle, in the apply's order."""
    return [(a, b) for a in range(P3) for b in range(a, P3)]


def test_stencil_counts_match_a_brute_force_count(bench):
    # p = 1 on a lattice: the assembled operator in difference form, the 26
    # off-diagonal coefficients of a row stored (the diagonal is implied)
    n = 7
    N, E, by, fl = bench.body_algorithmic(1, n)
    M = n + 1
    assert N == M ** 3 and E == n ** 3
    # rows x off-diagonal neighbour slots inside the lattice: what the
    # coefficient array holds beyond its zeros (boundary rows have fewer)
    inside = sum(1 for i in range(M) for j in range(M) for k in range(M)
                 for d in range(27) if d != 13
                 if 0 <= i + d % 3 - 1 < M and 0 <= j + (d // 3) % 3 - 1 < M and 0 <= k + d // 9 - 1 < M)
    assert inside == (3 * M - 2) ** 3 - N
    assert inside <= 26 * N
    assert by == 8 * 26 * N + 16 * N                  # coefficients, x, y
    assert fl == N * (3 * 26 + 2)                     # a difference and an FMA a term + x.y


@pytest.mark.parametrize("p", [2])
def test_element_matrix_counts_match_a_brute_force_count(bench, p):
    n = 7
    N, E, by, fl = bench.body_algorithmic(p, n)
    P3 = (p + 1) ** 3
    ent = packed_entries(P3)
    # y_e = K_e x_e from the upper triangle: one FMA on the diagonal, two off it
    fmas = sum(1 if a == b else 2 for a, b in ent)
    assert fmas == P3 * P3
    assert fl == E * (2 * fmas + 2 * P3)              # + x.y
    assert by == 16 * N + 4 * E * P3 + 8 * E * len(ent)
    assert E == n ** 3 and N == (p * n + 1) ** 3


@pytest.mark.parametrize("p", [3, 4, 8])
def test_sum_factorized_orders_keep_the_general_count(bench, p):
    assert bench.body_algorithmic(p, 5) == bench.algorithmic(p, 5)


def test_traffic_ratios_are_near_the_algorithmic_bytes(bench):
    # every order has a capture of its current default body, moving 1.0-1.2x
    # the algorithmic bytes (scattered y sectors, shared-node x re-reads, the
    # stencil's split pass), up to 1.4x where the body prefetches the next
    # group's qdata into L2 and part of it is evicted before use (p = 5, 6)
    # or spills registers to DRAM under its launch bound (p = 8)
    total = 0.0
    for p in range(1, 9):
        r = bench.dram_ratio(p)
        assert r is not None and 1.0 <= r <= (1.4 if p in (5, 6, 8) else 1.2), (p, r)
        n = fem_inputs.bp3_mesh_n(5e7, p)
        total += r * bench.body_algorithmic(p, n)[2]
    assert total > 0
