// Host-side cell-batch planning for the implicit cell passes (no CUDA): the
// cost-balanced cut of small meshes into one batch per persistent-solve CTA,
// and the cost-balanced order of many batches over the CTAs.  Header-only, so
// that a host test can compile it on its own.
#pragma once

#include <algorithm>
#include <cstdint>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

namespace dg {

// Batches of at most cpb consecutive cells, at most nb of them, with the
// largest batch cost as small as the greedy cut allows (bisection on the cost
// bound: each batch is closed when the next cell would exceed it or cpb is reached).
inline std::vector<int> balanced_batches(const std::vector<double>& cost, int cpb, int nb) {
  const int64_t K = (int64_t)cost.size();
  auto cut = [&](double bound, std::vector<int>* starts) {
    int count = 0, cells = 0;
    double acc = 0.0;
    for (int64_t c = 0; c < K; ++c) {
      if (cells > 0 && (cells == cpb || acc + cost[c] > bound)) {
        cells = 0;
        acc = 0.0;
      }
      if (cells == 0) {
        ++count;
        if (starts) starts->push_back((int)c);
      }
      acc += cost[c];
      ++cells;
    }
    return count;
  };
  double lo = *std::max_element(cost.begin(), cost.end()), hi = 0.0;
  for (double x : cost) hi += x;
  for (int it = 0; it < 60 && hi - lo > 1e-9 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (cut(mid, nullptr) <= nb) hi = mid;
    else lo = mid;
  }
  std::vector<int> starts;
  cut(hi, &starts);
  starts.push_back((int)K);
  return starts;
}

// An order of nb batches of costs bcost for G CTAs that take positions r,
// r + G, r + 2G, ... (order[position] = batch).  The first nb % G CTAs hold one
// position more than the others: they take the smallest batches there first;
// then the other batches, largest first, each go to the least loaded CTA with
// a position left.
inline std::vector<int> balanced_order(const std::vector<double>& bcost, int G) {
  const int nb = (int)bcost.size();
  const int q = nb / G, extra = nb % G;
  std::vector<int> idx(nb);
  for (int b = 0; b < nb; ++b) idx[b] = b;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return bcost[a] > bcost[b]; });
  std::vector<int> order(nb, -1);
  std::vector<double> load(G, 0.0);
  for (int r = 0; r < extra; ++r) {  // the extra positions (the last of those CTAs)
    const int b = idx[nb - extra + r];
    order[r + q * G] = b;
    load[r] = bcost[b];
  }
  using Slot = std::pair<double, int>;  // (load, CTA)
  std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
  std::vector<int> used(G, 0);
  if (q > 0)
    for (int r = 0; r < G; ++r) heap.push({load[r], r});
  for (int k = 0; k < nb - extra; ++k) {
    const int b = idx[k];
    const Slot sl = heap.top();
    heap.pop();
    const int r = sl.second;
    order[r + used[r] * G] = b;
    if (++used[r] < q) heap.push({sl.first + bcost[b], r});
  }
  return order;
}

}  // namespace dg
