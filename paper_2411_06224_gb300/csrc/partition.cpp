// Level-0 domain partition (Sec. 3.2, Eq. num_subdomains; supplement
// Algorithm 1), run once per mesh on the host like the paper's METIS step.
//
// METIS is replaced by recursive coordinate bisection of the rest
// positions: a set needing P = ceil(size / N) > 1 parts is split along the
// coordinate of largest extent (ties: x, then y, then z) into the first
// N * ceil(P / 2) nodes in (coordinate, index) order and the rest.  Leaves
// are numbered left to right, so every part but the last is full and
// M = ceil(n / N).  Node v then takes slot N * part + (rank of v among its
// part's nodes in ascending index), the paper's map array with padding.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gipc_mas_pcg.h"

namespace gs {
void set_error(const char* fmt, ...);
}

namespace {

struct Bisect {
  const double* X;
  int N;
  std::vector<int32_t> ids;
  std::vector<int32_t> part;
  int32_t next = 0;

  void run(size_t lo, size_t hi) {
    const size_t size = hi - lo;
    const size_t P = (size + N - 1) / N;
    if (P <= 1) {
      for (size_t i = lo; i < hi; ++i) part[ids[i]] = next;
      ++next;
      return;
    }
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (size_t i = lo; i < hi; ++i)
      for (int a = 0; a < 3; ++a) {
        const double v = X[3 * (size_t)ids[i] + a];
        mn[a] = std::min(mn[a], v);
        mx[a] = std::max(mx[a], v);
      }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
      if (mx[a] - mn[a] > mx[axis] - mn[axis]) axis = a;
    const size_t left = (size_t)N * ((P + 1) / 2);
    const double* Xp = X;
    auto less = [Xp, axis](int32_t u, int32_t v) {
      const double cu = Xp[3 * (size_t)u + axis], cv = Xp[3 * (size_t)v + axis];
      return cu < cv || (cu == cv && u < v);
    };
    std::nth_element(ids.begin() + lo, ids.begin() + lo + left, ids.begin() + hi, less);
    run(lo, lo + left);
    run(lo + left, hi);
  }
};

}  // namespace

extern "C" int gs_partition(int32_t n, const double* X, int32_t N, int32_t* map, int32_t* n_domains) {
  if (n <= 0 || !X || !map || !n_domains || N < 1) {
    gs::set_error("gs_partition: bad argument");
    return GS_ERR_INVALID;
  }
  for (int64_t i = 0; i < 3LL * n; ++i)
    if (!std::isfinite(X[i])) {
      gs::set_error("gs_partition: non-finite position");
      return GS_ERR_INVALID;
    }
  Bisect b;
  b.X = X;
  b.N = N;
  b.ids.resize(n);
  b.part.assign(n, -1);
  for (int32_t i = 0; i < n; ++i) b.ids[i] = i;
  b.run(0, (size_t)n);
  // rank inside each part in ascending node index
  std::vector<int32_t> fill(b.next, 0);
  for (int32_t v = 0; v < n; ++v) {
    const int32_t p = b.part[v];
    map[v] = p * N + fill[p]++;
  }
  *n_domains = b.next;
  return GS_OK;
}

// Several independent meshes, each partitioned on its own (no domain mixes
// two meshes): mesh s owns nodes [node_off[s], node_off[s+1]) and its parts
// follow those of mesh s-1.
extern "C" int gs_partition_batch(int32_t n_sys, const int32_t* node_off, const double* X, int32_t N, int32_t* map,
                                  int32_t* n_domains) {
  if (n_sys < 1 || !node_off || !X || !map || !n_domains || N < 1 || node_off[0] != 0) {
    gs::set_error("gs_partition_batch: bad argument");
    return GS_ERR_INVALID;
  }
  int32_t dom = 0;
  for (int32_t s = 0; s < n_sys; ++s) {
    const int32_t b = node_off[s], e = node_off[s + 1];
    if (e < b) {
      gs::set_error("gs_partition_batch: offsets not ascending");
      return GS_ERR_INVALID;
    }
    if (e == b) continue;
    int32_t nd = 0;
    int st = gs_partition(e - b, X + 3 * (int64_t)b, N, map + b, &nd);
    if (st != GS_OK) return st;
    for (int32_t v = b; v < e; ++v) map[v] += dom * N;
    dom += nd;
  }
  *n_domains = dom;
  return GS_OK;
}
