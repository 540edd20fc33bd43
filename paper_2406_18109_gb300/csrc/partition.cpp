// partition.cpp -- host-side plans over a CSR matrix: its row-block
// partition over ranks, and the x windows each SpMV point reads.
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
// The second plan (dfs_spmv_windows, at the end) lists, for each tile of
// rows, the intervals of x its rows read, for kernels that stage them in
// shared memory.
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

// ------------------------------------------------------ SpMV x windows
// For each point of an SpMV (a tile of rows), the columns its rows read,
// as at most three intervals of x widened to 16-byte boundaries: the data a
// kernel copies into shared memory before the rows run (see DFS_OP_SPMV).
extern "C" int dfs_spmv_windows(const int32_t* rowptr, const int32_t* col, int64_t nrows, int64_t ncols,
                                int64_t tile, int32_t elem_bytes, int64_t budget_bytes, int32_t* out) {
  if (!rowptr || !out || nrows < 0 || ncols < 0 || ncols > INT32_MAX || tile < 1 ||
      (elem_bytes != 4 && elem_bytes != 8) || rowptr[0] != 0)
    return DFS_ERR_INVALID;
  for (int64_t i = 0; i < nrows; ++i)
    if (rowptr[i + 1] < rowptr[i]) return DFS_ERR_INVALID;
  if (rowptr[nrows] > 0 && !col) return DFS_ERR_INVALID;
  for (int64_t k = 0; k < rowptr[nrows]; ++k)
    if (col[k] < 0 || col[k] >= ncols) return DFS_ERR_INVALID;
  const int64_t q = 16 / elem_bytes;             // elements per 16 bytes
  const int64_t end_al = ncols / q * q;          // the aligned part of [0, ncols)
  const int64_t npts = (nrows + tile - 1) / tile;
  std::vector<int32_t> cs;
  std::vector<std::pair<int64_t, int64_t>> iv;
  for (int64_t p = 0; p < npts; ++p) {
    int32_t* rec = out + 6 * p;
    for (int k = 0; k < 6; ++k) rec[k] = 0;
    const int64_t r0 = p * tile, r1 = std::min(r0 + tile, nrows);
    cs.assign(col + rowptr[r0], col + rowptr[r1]);
    std::sort(cs.begin(), cs.end());
    cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
    iv.clear();
    for (int32_t c : cs) {
      if (!iv.empty() && c <= iv.back().second + 64) iv.back().second = (int64_t)c + 1;
      else iv.push_back({c, (int64_t)c + 1});
    }
    while (iv.size() > 3) {  // merge the two intervals with the smallest gap
      size_t best = 0;
      for (size_t k = 1; k + 1 < iv.size(); ++k)
        if (iv[k + 1].first - iv[k].second < iv[best + 1].first - iv[best].second) best = k;
      iv[best].second = iv[best + 1].second;
      iv.erase(iv.begin() + (int64_t)best + 1);
    }
    // widen to 16-byte boundaries, clip to the aligned part of x, merge overlaps
    std::vector<std::pair<int64_t, int64_t>> al;
    for (const auto& v : iv) {
      const int64_t lo = v.first / q * q;
      const int64_t hi = std::min((v.second + q - 1) / q * q, end_al);
      if (hi <= lo) continue;
      if (!al.empty() && lo <= al.back().second) al.back().second = std::max(al.back().second, hi);
      else al.push_back({lo, hi});
    }
    int64_t tot = 0;
    for (const auto& v : al) tot += v.second - v.first;
    if (al.empty() || tot * elem_bytes > budget_bytes) continue;
    for (size_t k = 0; k < al.size(); ++k) {
      rec[2 * k] = (int32_t)al[k].first;
      rec[2 * k + 1] = (int32_t)(al[k].second - al[k].first);
    }
  }
  return DFS_OK;
}
