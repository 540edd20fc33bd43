// partition.cpp -- row-block partition of a CSR matrix over ranks (host only).
//
// Section 3.2: an index task's launch domain is split into point tasks, one
// per processor; across GPUs a vector store is tiled by row blocks and every
// point task owns one block.  A CSR SpMV task reads x through the None
// partition (any row may touch any column), so a point task whose rows touch
// columns of another block needs those entries of x before it runs: the
// HALO.  This file computes, for one rank, which global rows it owns, its
// rows renumbered to local columns (owned entries first, halo slots after),
// the halo slots it receives from each rank and the owned entries it sends to
// each rank.  The exchange itself and the solver steps run elsewhere.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "../../include/diffuse.h"

namespace {

void bounds(int64_t n, int32_t nranks, int32_t r, int64_t* lo, int64_t* hi) {
  // balanced blocks: rank r owns [floor(r n / P), floor((r + 1) n / P))
  *lo = (int64_t)((__int128)n * r / nranks);
  *hi = (int64_t)((__int128)n * (r + 1) / nranks);
}

// Owner of global row g under the balanced blocks (the inverse of bounds).
int32_t owner(int64_t g, int64_t n, int32_t nranks) {
  int32_t q = (int32_t)((__int128)(g + 1) * nranks / n);   // first guess, then step to the block
  if (q >= nranks) q = nranks - 1;
  int64_t lo, hi;
  for (;;) {
    bounds(n, nranks, q, &lo, &hi);
    if (g < lo) --q;
    else if (g >= hi) ++q;
    else return q;
  }
}

int check(const int32_t* rowptr, const int32_t* col, int64_t n, int32_t nranks, int32_t rank) {
  if (n < 0 || nranks < 1 || rank < 0 || rank >= nranks || !rowptr || (n > 0 && !col && rowptr[n] > 0))
    return DFS_ERR_INVALID;
  if (n > INT32_MAX || rowptr[0] != 0) return DFS_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return DFS_ERR_INVALID;
  for (int64_t k = 0; k < rowptr[n]; ++k)
    if (col[k] < 0 || col[k] >= n) return DFS_ERR_INVALID;
  return DFS_OK;
}

struct Plan {
  int64_t lo = 0, hi = 0;
  std::vector<int64_t> halo;                    // global columns, ascending
  std::vector<int64_t> recv_counts, send_counts;
  std::vector<int32_t> send_idx;                // local owned indices, grouped by destination
};

Plan make_plan(const int32_t* rowptr, const int32_t* col, int64_t n, int32_t nranks, int32_t rank) {
  Plan p;
  bounds(n, nranks, rank, &p.lo, &p.hi);
  p.recv_counts.assign(nranks, 0);
  p.send_counts.assign(nranks, 0);
  // halo: distinct columns of the owned rows outside [lo, hi); ascending
  // global order groups them by owner rank, since blocks are contiguous
  for (int64_t i = p.lo; i < p.hi; ++i)
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] < p.lo || col[k] >= p.hi) p.halo.push_back(col[k]);
  std::sort(p.halo.begin(), p.halo.end());
  p.halo.erase(std::unique(p.halo.begin(), p.halo.end()), p.halo.end());
  for (int64_t g : p.halo) ++p.recv_counts[owner(g, n, nranks)];
  // sends: for every other rank q, the owned entries its rows read, ascending
  // (q's halo slots from this rank are in the same ascending global order)
  std::vector<int32_t> mark;
  for (int32_t q = 0; q < nranks; ++q) {
    if (q == rank) continue;
    int64_t qlo, qhi;
    bounds(n, nranks, q, &qlo, &qhi);
    mark.clear();
    for (int64_t i = qlo; i < qhi; ++i)
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
        if (col[k] >= p.lo && col[k] < p.hi) mark.push_back((int32_t)(col[k] - p.lo));
    std::sort(mark.begin(), mark.end());
    mark.erase(std::unique(mark.begin(), mark.end()), mark.end());
    p.send_counts[q] = (int64_t)mark.size();
    p.send_idx.insert(p.send_idx.end(), mark.begin(), mark.end());
  }
  return p;
}

}  // namespace

extern "C" int dfs_rowblock_bounds(int64_t n, int32_t nranks, int32_t rank, int64_t* lo, int64_t* hi) {
  if (n < 0 || nranks < 1 || rank < 0 || rank >= nranks || !lo || !hi) return DFS_ERR_INVALID;
  bounds(n, nranks, rank, lo, hi);
  return DFS_OK;
}

extern "C" int dfs_rowblock_sizes(const int32_t* rowptr, const int32_t* col, int64_t n, int32_t nranks,
                                  int32_t rank, dfs_rowblock_sizes_t* out) {
  if (!out) return DFS_ERR_INVALID;
  const int rc = check(rowptr, col, n, nranks, rank);
  if (rc) return rc;
  const Plan p = make_plan(rowptr, col, n, nranks, rank);
  out->row_lo = p.lo;
  out->row_hi = p.hi;
  out->nnz = (int64_t)rowptr[p.hi] - rowptr[p.lo];
  out->n_halo = (int64_t)p.halo.size();
  out->n_send = (int64_t)p.send_idx.size();
  return DFS_OK;
}

extern "C" int dfs_rowblock_plan(const int32_t* rowptr, const int32_t* col, int64_t n, int32_t nranks,
                                 int32_t rank, int32_t* local_rowptr, int32_t* local_col, int64_t* halo_cols,
                                 int64_t* recv_counts, int32_t* send_idx, int64_t* send_counts) {
  const int rc = check(rowptr, col, n, nranks, rank);
  if (rc) return rc;
  if (!local_rowptr || !recv_counts || !send_counts) return DFS_ERR_INVALID;
  const Plan p = make_plan(rowptr, col, n, nranks, rank);
  const int64_t n_own = p.hi - p.lo;
  const int64_t nnz = (int64_t)rowptr[p.hi] - rowptr[p.lo];
  if ((nnz > 0 && !local_col) || (!p.halo.empty() && !halo_cols) || (!p.send_idx.empty() && !send_idx))
    return DFS_ERR_INVALID;
  if (n_own + (int64_t)p.halo.size() > INT32_MAX) return DFS_ERR_TOO_LARGE;
  for (int64_t i = 0; i <= n_own; ++i) local_rowptr[i] = rowptr[p.lo + i] - rowptr[p.lo];
  for (int64_t k = 0; k < nnz; ++k) {
    const int64_t g = col[rowptr[p.lo] + k];
    if (g >= p.lo && g < p.hi) {
      local_col[k] = (int32_t)(g - p.lo);
    } else {
      const int64_t slot = std::lower_bound(p.halo.begin(), p.halo.end(), g) - p.halo.begin();
      local_col[k] = (int32_t)(n_own + slot);
    }
  }
  std::copy(p.halo.begin(), p.halo.end(), halo_cols);
  std::copy(p.recv_counts.begin(), p.recv_counts.end(), recv_counts);
  std::copy(p.send_idx.begin(), p.send_idx.end(), send_idx);
  std::copy(p.send_counts.begin(), p.send_counts.end(), send_counts);
  return DFS_OK;
}
