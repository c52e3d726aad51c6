"""Host planning of the implicit passes' cell batches (csrc/partition.h), compiled on its own with
the host C++ compiler: the cost-balanced cut of a small mesh into batches of at most CPB
consecutive cells, one per CTA of a persistent solve, and the cost-balanced order of a large mesh's
batches over the CTAs (CTA r taking positions r, r + G, ...).  No GPU."""

import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(HERE, "..", "paper_2408_08129_gb300", "csrc", "partition.h")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "partition.h"
int main() {
  int mode, n, a, b;
  while (std::scanf("%d %d %d %d", &mode, &n, &a, &b) == 4) {
    std::vector<double> c(n);
    for (int i = 0; i < n; ++i) std::scanf("%lf", &c[i]);
    const std::vector<int> r = mode == 0 ? dg::balanced_batches(c, a, b) : dg::balanced_order(c, a);
    std::printf("%zu", r.size());
    for (int x : r) std::printf(" %d", x);
    std::printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("partition")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)], check=True)

    def run(mode, costs, a, b=0):
        inp = "%d %d %d %d\n%s\n" % (mode, len(costs), a, b, " ".join("%.17g" % x for x in costs))
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split()
        m = int(out[0])
        return [int(x) for x in out[1:1 + m]]

    return run


def _optimal_max(costs, cpb, nb):
    """Smallest possible largest batch cost over cuts into at most nb batches of at most cpb
    consecutive cells (dynamic programming over cut positions)."""
    K = len(costs)
    pre = np.concatenate([[0.0], np.cumsum(costs)])
    INF = float("inf")
    best = [[INF] * (nb + 1) for _ in range(K + 1)]  # best[i][j]: first i cells in j batches
    best[0][0] = 0.0
    for i in range(1, K + 1):
        for j in range(1, nb + 1):
            for s in range(max(0, i - cpb), i):
                if best[s][j - 1] < INF:
                    best[i][j] = min(best[i][j], max(best[s][j - 1], pre[i] - pre[s]))
    return min(best[K][1:])


@pytest.mark.parametrize("seed,K,cpb,nb", [(0, 37, 5, 12), (1, 60, 10, 9), (2, 25, 3, 25), (3, 48, 8, 7),
                                           (4, 11, 4, 3)])
def test_balanced_cut_is_a_valid_optimal_cut(planner, seed, K, cpb, nb):
    rng = np.random.default_rng(seed)
    costs = 25.0 + rng.integers(0, 4, K) * rng.uniform(5.0, 40.0, K)  # plain cells, some with 2:1 faces
    starts = planner(0, costs, cpb, nb)
    assert starts[0] == 0 and starts[-1] == K
    sizes = np.diff(starts)
    assert (sizes >= 1).all() and (sizes <= cpb).all()
    assert len(sizes) <= nb
    worst = max(costs[s:e].sum() for s, e in zip(starts[:-1], starts[1:]))
    assert worst <= _optimal_max(costs, cpb, nb) * (1 + 1e-6)


def test_balanced_cut_of_uniform_cells_is_even(planner):
    starts = planner(0, [1.0] * 100, 10, 20)
    assert sorted(set(np.diff(starts))) == [5]


def _loads(costs, order, G):
    loads = np.zeros(G)
    for p, b in enumerate(order):
        loads[p % G] += costs[b]
    return loads


@pytest.mark.parametrize("seed,nb,G", [(0, 1000, 304), (1, 986, 304), (2, 305, 304), (3, 47, 8), (4, 7, 8)])
def test_balanced_order_is_a_permutation_that_evens_the_ctas(planner, seed, nb, G):
    rng = np.random.default_rng(seed)
    costs = 250.0 + (rng.random(nb) < 0.1) * rng.uniform(50.0, 400.0, nb)  # a tenth hold coarse sides
    order = planner(1, costs, G)
    assert sorted(order) == list(range(nb))
    lpt = _loads(costs, order, G).max()
    plain = _loads(costs, list(range(nb)), G).max()
    assert lpt <= plain + 1e-9
    # every CTA gets floor or ceil of nb / G batches, so the heaviest one carries at most that many
    # of the largest costs
    per = -(-nb // G)
    assert lpt <= np.sort(costs)[::-1][:per].sum() + 1e-9


def test_balanced_order_of_equal_costs_is_the_identity_load(planner):
    order = planner(1, [3.0] * 20, 8)
    loads = _loads([3.0] * 20, order, 8)
    assert sorted(set(loads)) == [6.0, 9.0]
