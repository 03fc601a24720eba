// The work list of the enumeration kernel: subset prefixes split until small enough, in
// lexicographic order, and their grouping into ranges (host side; plain C++17).
#include <algorithm>
#include <vector>

#include "bd_host.h"

namespace bd {

namespace {

// a 5-D node (depth K-3) is split by its quadruples' first point when it holds more than this
// many times the split threshold
constexpr uint64_t kNodeSplit = 16;

// every prefix of the split tree, depth first; emit(item) returns false to stop early
template <class Emit>
bool for_each_item(int N, int K, uint64_t max_subsets, int depth, Emit emit) {
  if (K < 1 || N < K + 1) return true;
  int pre[KMAX + 1];
  int len = 1;
  pre[0] = 0;
  for (;;) {
    const uint64_t T = subtree_size(N, K, pre[len - 1], len);
    // split; items stop where the bottom stage starts, except that a node of the 5-D stage much
    // larger than the threshold splits once more, by the first point of its quadruples, so
    // that no single node holds a large share of a launch
    const bool split = len < depth ? T > max_subsets
                                   : depth == K - 3 && K >= 4 && len == depth && T / kNodeSplit > max_subsets;
    if (split) {
      pre[len] = pre[len - 1] + 1;
      ++len;
      continue;
    }
    if (T > 0) {
      Item x{};
      x.len = (uint8_t)len;
      for (int i = 0; i < len; ++i) x.idx[i] = (uint8_t)pre[i];
      if (!emit(x)) return false;
    }
    // next sibling, backtracking as needed; position i admits indices up to N-1-(K-i)
    for (;;) {
      const int nxt = pre[len - 1] + 1;
      if (nxt <= N - 1 - (K - (len - 1))) { pre[len - 1] = nxt; break; }
      if (--len == 0) return true;
    }
  }
}

// largest subtree first; ties broken by the prefix itself, so the order is a total order (the
// same order build_items produces; used where no allocation is allowed)
struct ItemOrder {
  int N, K;
  bool operator()(const Item& a, const Item& b) const {
    const uint64_t sa = subtree_size(N, K, a.idx[a.len - 1], a.len), sb = subtree_size(N, K, b.idx[b.len - 1], b.len);
    if (sa != sb) return sa > sb;
    if (a.len != b.len) return a.len < b.len;
    for (int i = 0; i < a.len; ++i)
      if (a.idx[i] != b.idx[i]) return a.idx[i] < b.idx[i];
    return false;
  }
};

}  // namespace

bool prefer_five(const int64_t* points, int npts, int k, uint64_t teams) {
  if (k < 4 || k > KMAX || npts < k + 1 || npts > NMAX) return false;
  if (teams == 0) return true;
  if (k < 6) return false;
  constexpr int kSamples = 256;
  uint64_t z = 0x243F6A8885A308D3ull ^ ((uint64_t)npts << 32 | (uint64_t)k);
  auto next = [&z]() {  // SplitMix64 step
    z += 0x9E3779B97F4A7C15ull;
    uint64_t x = z;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
  };
  int idx[NMAX];
  int64_t M[KMAX][KMAX];
  int full = 0;
  for (int t = 0; t < kSamples; ++t) {
    for (int i = 0; i < npts; ++i) idx[i] = i;
    for (int i = 0; i <= k; ++i) {  // a uniform (k+1)-subset: partial Fisher-Yates
      const int j = i + (int)(next() % (uint64_t)(npts - i));
      std::swap(idx[i], idx[j]);
    }
    for (int r = 0; r < k; ++r)
      for (int c = 0; c < k; ++c) M[r][c] = points[(size_t)idx[r + 1] * k + c] - points[(size_t)idx[0] * k + c];
    // fraction-free elimination: every entry stays a minor of the differences, below 2^31 on the
    // 32-bit coordinate path (the only one that asks), so products fit 64 bits; divisions exact
    int64_t prev = 1;
    bool nonsingular = true;
    for (int p = 0; p < k && nonsingular; ++p) {
      int r = p;
      while (r < k && M[r][p] == 0) ++r;
      if (r == k) {
        nonsingular = false;
        break;
      }
      if (r != p)
        for (int c = 0; c < k; ++c) std::swap(M[r][c], M[p][c]);
      for (int i = p + 1; i < k; ++i) {
        for (int c = p + 1; c < k; ++c)
          M[i][c] = (M[i][c] * M[p][p] - M[i][p] * M[p][c]) / prev;
        M[i][p] = 0;
      }
      prev = M[p][p];
    }
    full += nonsingular ? 1 : 0;
    // a clear majority after 64 or 128 samples decides (the rule only steers speed)
    if ((t + 1 == 64 || t + 1 == 128) && (full * 20 <= (t + 1) * 7 || full * 20 >= (t + 1) * 13)) return full * 2 <= t + 1;
  }
  return full * 2 <= kSamples;
}

int item_depth(int K, int path, bool five) { return five && K >= 4 && path == 0 ? K - 3 : std::max(K - 2, 1); }

std::vector<Item> build_items(int N, int K, uint64_t max_subsets, int depth, bool sorted) {
  std::vector<Item> items;
  std::vector<uint64_t> size;
  for_each_item(N, K, max_subsets, depth, [&](const Item& x) {
    items.push_back(x);
    size.push_back(subtree_size(N, K, x.idx[x.len - 1], x.len));
    return true;
  });
  if (!sorted) return items;
  // largest subtree first, then shorter prefixes; items of equal size and length keep their
  // lexicographic generation order (a stable sort), so the order is a total order
  std::vector<uint32_t> ord(items.size());
  for (uint32_t i = 0; i < ord.size(); ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) {
    if (size[a] != size[b]) return size[a] > size[b];
    return items[a].len < items[b].len;
  });
  std::vector<Item> out(items.size());
  for (size_t i = 0; i < ord.size(); ++i) out[i] = items[ord[i]];
  return out;
}

// estimated work of an item, in warp rounds of the bottom stage plus one per level step
static uint64_t item_cost(int N, int K, int D, const Item& it) {
  const int L = it.len, a = it.idx[L - 1];
  if (K < 3) return subtree_size(N, K, a, L);
  // the bottom stage runs on nodes of depth D with R points after their last index: the 5-D
  // test (D = K-3) takes one Bareiss step, ceil(C(R,4)/32) warp rounds and about one round of
  // queued quadruples, the 4-D test (D = K-2) one step and ceil(C(R,3)/32) rounds; nodes with
  // last index v below this prefix: C(v-a-1, D-1-L) (none deeper when L = D)
  const bool five = D == K - 3;
  const int m = five ? 4 : 3;
  auto node = [&](int v) {
    const uint64_t t = binom(N - 1 - v, m);
    return (uint64_t)(five ? 2 : 1) + (t + 31) / 32;
  };
  if (L > D) return 1 + (binom(N - 1 - a, 3) + 31) / 32;  // a 5-D item below its node
  if (L == D) return node(a);
  uint64_t c = 0;
  for (int v = a + (D - L); v <= N - 1 - m; ++v) c += binom(v - a - 1, D - 1 - L) * node(v);
  return c;
}

uint64_t default_item_subsets(uint64_t total, uint64_t teams) {
  const uint64_t t = total / (teams * 32 + 1);
  return std::min<uint64_t>(std::max<uint64_t>(t, 64), (uint64_t)1 << 20);
}

void build_ranges(int N, int K, uint64_t max_subsets, uint64_t teams, int depth, std::vector<Item>& items,
                  std::vector<Range>& ranges) {
  items.clear();
  ranges.clear();
  std::vector<uint64_t> cost;
  uint64_t remaining = 0;
  for_each_item(N, K, max_subsets, depth, [&](const Item& x) {
    items.push_back(x);
    cost.push_back(std::max<uint64_t>(1, item_cost(N, K, depth, x)));
    remaining += cost.back();
    return true;
  });
  // runs of consecutive items packed up to 1/8 of a team's share, then taken largest first
  const uint64_t cap = std::max<uint64_t>(1, remaining / (8 * std::max<uint64_t>(1, teams)));
  std::vector<uint64_t> rcost;
  size_t i = 0;
  while (i < items.size()) {
    const size_t first = i;
    uint64_t got = 0;
    while (i < items.size() && (i == first || got + cost[i] <= cap)) got += cost[i++];
    ranges.push_back(Range{(uint32_t)first, (uint32_t)(i - first)});
    rcost.push_back(got);
  }
  std::vector<size_t> order(ranges.size());
  for (size_t r = 0; r < order.size(); ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return rcost[a] > rcost[b]; });
  std::vector<Range> sorted;
  sorted.reserve(ranges.size());
  for (size_t r : order) sorted.push_back(ranges[r]);
  ranges.swap(sorted);
}

bool build_items_into(int N, int K, uint64_t max_subsets, int depth, Item* out, size_t cap, size_t* count) {
  size_t n = 0;
  const bool ok = for_each_item(N, K, max_subsets, depth, [&](const Item& x) {
    if (n == cap) return false;
    out[n++] = x;
    return true;
  });
  *count = n;
  if (!ok) return false;
  std::sort(out, out + n, ItemOrder{N, K});
  return true;
}

}  // namespace bd
