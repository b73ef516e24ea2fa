// HQR elimination-list generator and validator (host C++).
//
// Sec. 4.1-4.2 compose the list from per-panel reduction trees: TS domains of
// `a` tiles (level 0), a low-level tree over the TS heads of each of the p
// virtual domains (level 1), optionally the coupling ("domino") level
// (level 2), and a high-level tree over the domain tops (level 3). Tree shapes follow Sec. 3.1 (flat, binary), Sec. 3.2 (greedy,
// Table 4) and the Modi-Clarke "Fibonacci" scheme that Sec. 3.3 names.
// Steps follow the unit-time model of Sec. 3.1-3.2.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/hqr.h"

namespace {

struct Pair {
  int killed, killer;
};

// Flat tree (Sec. 3.1): the first leaf kills the others, top to bottom.
void flat_tree(const std::vector<int> &leaves, std::vector<Pair> &out) {
  for (size_t q = 1; q < leaves.size(); ++q) out.push_back({leaves[q], leaves[0]});
}

// Binary tree (Sec. 3.1): at distance d = 1, 2, 4, ... leaf j kills leaf
// j + d for every j that is a multiple of 2d.
void binary_tree(const std::vector<int> &leaves, std::vector<Pair> &out) {
  const int R = (int)leaves.size();
  for (int d = 1; d < R; d *= 2)
    for (int j = 0; j + d < R; j += 2 * d) out.push_back({leaves[j + d], leaves[j]});
}

// Fibonacci (Modi-Clarke order 1). With x the least integer such that
// x(x+1)/2 >= R-1, leaf positions 1..R-1 are cut from the top into groups
// of 1, 2, 3, ... positions (the last one truncated). Group g (planned step
// x-g+1) is killed by as many leaves as it holds, taken right above it, in
// natural order. Emitted in planned-step order: largest g first.
void fibonacci_tree(const std::vector<int> &leaves, std::vector<Pair> &out) {
  const int R = (int)leaves.size();
  if (R <= 1) return;
  struct G {
    int start, end;
  };
  std::vector<G> groups;
  for (int start = 1, g = 1; start < R; ++g) {
    int end = std::min(start + g, R);
    groups.push_back({start, end});
    start = end;
  }
  for (int q = (int)groups.size() - 1; q >= 0; --q) {
    const int s = groups[q].end - groups[q].start;
    for (int t = 0; t < s; ++t)
      out.push_back({leaves[groups[q].start + t], leaves[groups[q].start - s + t]});
  }
}

struct Emit {
  int killed, killer, step;
};

// Greedy with readiness (Sec. 3.2): at time t, the alive leaves whose last
// elimination is before t are candidates (ascending); the bottom half (floor)
// is killed by the same number of candidates right above, in natural order.
void greedy_tree(const std::vector<int> &leaves, std::vector<int> &busy,
                 std::vector<Emit> &out) {
  std::vector<int> alive(leaves);
  if (alive.size() <= 1) return;
  int t = busy[alive[0]];
  for (int r : alive) t = std::min(t, busy[r]);
  t += 1;
  std::vector<int> cand;
  std::vector<char> dead;
  while (alive.size() > 1) {
    cand.clear();
    for (int r : alive)
      if (busy[r] < t) cand.push_back(r);
    const int z = (int)cand.size() / 2;
    if (z > 0) {
      const int c = (int)cand.size();
      for (int q = 0; q < z; ++q) {
        const int kd = cand[c - z + q], kr = cand[c - 2 * z + q];
        out.push_back({kd, kr, t});
        busy[kd] = t;
        busy[kr] = t;
      }
      std::vector<int> keep;
      keep.reserve(alive.size());
      // the killed rows are exactly cand[c-z .. c-1]
      size_t w = (size_t)(c - z);
      for (int r : alive) {
        if (w < cand.size() && r == cand[w]) {
          ++w;
          continue;
        }
        keep.push_back(r);
      }
      alive.swap(keep);
    }
    ++t;
  }
}

void run_tree(int tree, const std::vector<int> &leaves, std::vector<int> &busy,
              std::vector<Emit> &out) {
  if (tree == HQR_GREEDY) {
    greedy_tree(leaves, busy, out);
    return;
  }
  std::vector<Pair> pairs;
  if (tree == HQR_FLAT)
    flat_tree(leaves, pairs);
  else if (tree == HQR_BINARY)
    binary_tree(leaves, pairs);
  else
    fibonacci_tree(leaves, pairs);
  for (const Pair &pr : pairs) {
    const int step = std::max(busy[pr.killed], busy[pr.killer]) + 1;
    busy[pr.killed] = step;
    busy[pr.killer] = step;
    out.push_back({pr.killed, pr.killer, step});
  }
}

}  // namespace

namespace {

// The list of Sec. 4.1-4.2. In panel k the active rows of domain c are its
// rows >= k; its top is the first of them. Without the coupling level the TS
// domains and the low-level tree reduce all active rows to the top. With it
// (Sec. 4.2, level 2) they reduce only the rows on and below the domain's
// local diagonal (local index k, row k p + c), whose survivor is that
// diagonal row; the rows between the top and the local diagonal (the
// diagonal row included) are then killed by the top, one after the other in
// ascending order, with TT kernels (the domino tree).
int elim_list(int m, int n, int a, int p, int low_tree, int high_tree, bool domino, hqr_elim_t *out,
              size_t cap, size_t *count) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (a < 1) return -3;
  if (p < 1) return -4;
  if (low_tree < 0 || low_tree > 3) return -5;
  if (high_tree < 0 || high_tree > 3) return -6;
  if (!count) return -9;
  size_t need = 0;
  for (int k = 0; k < n; ++k) need += (size_t)(m - k - 1);
  *count = need;
  if (cap < need) return HQR_ERR_CAPACITY;
  if (need > 0 && !out) return -7;

  std::vector<int> busy(m, 0);
  std::vector<hqr_elim_t> panel;
  std::vector<int> rows, local, coupled, heads, tops;
  std::vector<Emit> em;
  size_t pos = 0;
  for (int k = 0; k < n; ++k) {
    panel.clear();
    tops.clear();
    for (int c = 0; c < p; ++c) {
      rows.clear();
      // first row >= k in domain c (rows congruent to c mod p)
      int first = k + ((c - k % p) % p + p) % p;
      for (int i = first; i < m; i += p) rows.push_back(i);
      if (rows.empty()) continue;
      const int top = rows[0];
      const long long base = domino ? (long long)k * p + c : top;  // first row of the local reduction
      local.clear();
      coupled.clear();
      for (int i : rows) {
        if (i >= base)
          local.push_back(i);
        else if (i > top)
          coupled.push_back(i);
      }
      if (!local.empty() && local[0] != top) coupled.push_back(local[0]);  // the local survivor
      heads.clear();
      for (size_t h = 0; h < local.size(); h += (size_t)a) {
        heads.push_back(local[h]);
        const int head = local[h];
        for (size_t q = h + 1; q < h + (size_t)a && q < local.size(); ++q) {
          const int i = local[q];
          const int step = std::max(busy[i], busy[head]) + 1;
          busy[i] = step;
          busy[head] = step;
          panel.push_back({k, i, head, HQR_KIND_TS, 0, step});
        }
      }
      em.clear();
      run_tree(low_tree, heads, busy, em);
      for (const Emit &e : em) panel.push_back({k, e.killed, e.killer, HQR_KIND_TT, 1, e.step});
      for (int i : coupled) {  // level 2: the top kills the coupled rows in ascending order
        const int step = std::max(busy[i], busy[top]) + 1;
        busy[i] = step;
        busy[top] = step;
        panel.push_back({k, i, top, HQR_KIND_TT, 2, step});
      }
      tops.push_back(top);
    }
    std::sort(tops.begin(), tops.end());
    em.clear();
    run_tree(high_tree, tops, busy, em);
    for (const Emit &e : em) panel.push_back({k, e.killed, e.killer, HQR_KIND_TT, 3, e.step});
    std::sort(panel.begin(), panel.end(), [](const hqr_elim_t &x, const hqr_elim_t &y) {
      return x.step != y.step ? x.step < y.step : x.i < y.i;
    });
    for (const hqr_elim_t &r : panel) out[pos++] = r;
  }
  return pos == need ? HQR_SUCCESS : HQR_ERR_INTERNAL;
}

}  // namespace

extern "C" int hqr_elim_list(int m, int n, int a, int p, int low_tree, int high_tree,
                             hqr_elim_t *out, size_t cap, size_t *count) {
  return elim_list(m, n, a, p, low_tree, high_tree, false, out, cap, count);
}

extern "C" int hqr_elim_list_domino(int m, int n, int a, int p, int low_tree, int high_tree,
                                    hqr_elim_t *out, size_t cap, size_t *count) {
  return elim_list(m, n, a, p, low_tree, high_tree, true, out, cap, count);
}

extern "C" int hqr_validate_list(int m, int n, const hqr_elim_t *list, size_t count) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (count > 0 && !list) return -3;
  const int K = std::min(m, n);
  // position of the record that kills (i, k); -1 = none yet
  std::vector<long long> pos((size_t)m * K, -1);
  for (size_t q = 0; q < count; ++q) {
    const hqr_elim_t &r = list[q];
    if (r.k < 0 || r.k >= K) return HQR_ERR_INVALID_LIST;
    if (r.i <= r.k || r.i >= m) return HQR_ERR_INVALID_LIST;
    if (r.killer < r.k || r.killer >= m || r.killer == r.i) return HQR_ERR_INVALID_LIST;
    if (r.kind != HQR_KIND_TS && r.kind != HQR_KIND_TT) return HQR_ERR_INVALID_LIST;
    long long &p = pos[(size_t)r.k * m + r.i];
    if (p >= 0) return HQR_ERR_INVALID_LIST;  // killed twice
    p = (long long)q;
  }
  for (int k = 0; k < K; ++k)
    for (int i = k + 1; i < m; ++i)
      if (pos[(size_t)k * m + i] < 0) return HQR_ERR_INVALID_LIST;  // never killed
  for (size_t q = 0; q < count; ++q) {
    const hqr_elim_t &r = list[q];
    for (int kp = 0; kp < r.k; ++kp) {
      if (r.i > kp && pos[(size_t)kp * m + r.i] > (long long)q) return HQR_ERR_INVALID_LIST;
      if (r.killer > kp && pos[(size_t)kp * m + r.killer] > (long long)q)
        return HQR_ERR_INVALID_LIST;
    }
    if (r.killer > r.k && pos[(size_t)r.k * m + r.killer] < (long long)q)
      return HQR_ERR_INVALID_LIST;  // killer already zeroed
  }
  // tile states within a panel: a TS victim must be square (never a killer
  // before), and a TS-zeroed row cannot kill.
  std::vector<int> state(m);  // 0 square, 1 triangle, 2 zero
  for (int k = 0; k < K; ++k) {
    std::fill(state.begin(), state.end(), 0);
    for (size_t q = 0; q < count; ++q) {
      const hqr_elim_t &r = list[q];
      if (r.k != k) continue;
      if (state[r.killer] == 2) return HQR_ERR_INVALID_LIST;
      if (r.kind == HQR_KIND_TS && state[r.i] != 0) return HQR_ERR_INVALID_LIST;
      state[r.killer] = 1;
      state[r.i] = 2;
    }
  }
  return HQR_SUCCESS;
}
