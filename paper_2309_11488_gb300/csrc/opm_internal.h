// Internal declarations of the GB300 BSR ILU0-BiCGStab library.
//
// Device data layout ("warp-sliced" block storage, used for A, L and U):
//   Rows are in the schedule's order and grouped in slices of 32 consecutive
//   rows, one slice per warp, one row per lane.  The blocks of a slice occupy
//   the same block range as in CSR (rowptr[32s] .. rowptr[32s+32]) but are
//   reordered "k-major": slab k holds the k-th block of every row of the slice
//   that has more than k blocks, in lane order.  Inside slab k the 9 entries
//   are stored entry-planar: entry e of the block of rank q is value
//   9*base_k + e*cnt_k + q, where base_k is the slab's first block and cnt_k
//   its number of blocks.  A warp walking slab k therefore reads every entry
//   with one coalesced load, and the storage has no padding.  A lane finds
//   cnt_k = popc(ballot(len > k)) and q = popc(ballot & lanemask_lt) itself,
//   so only the CSR row pointer is needed to walk a row.
//
//   In A's layout a row's diagonal block comes first, then the others in
//   column order (L and U layouts: column order).
//
//   A "slot" packs the location of one block: (entry-0 value index << 6) |
//   stride, with stride = cnt_k <= 32; entry e lives at off + e*stride.
//
//   The inverted diagonal blocks of U (Dinv) are stored per slice as 9 planes
//   of 32 values: row i's entry e is value 288*(i/32) + 32*e + i%32.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/opm_bsr.h"

namespace opm {

constexpr int kWarp = 32;
constexpr int kTileRows = 1024;    // rows per tile of the streaming kernels (256 threads x 4)
constexpr int kSpmvRows = 256;     // rows per tile of the SpMV kernels (256 threads x 1)
constexpr int kSweepThreads = 1024;  // threads per CTA of the cooperative sweep kernels
constexpr int kSliceVals = 288;  // 32 rows x 9 entries per Dinv slice
constexpr int32_t kRunning = 0x7fffffff;

inline int64_t slot_pack(int64_t off, int stride) { return (off << 6) | (int64_t)stride; }

// Result of the host symbolic analysis of one pattern (Section 4.4).
struct Analysis {
  int32_t n = 0;
  int64_t nnzb = 0, nnz_l = 0, nnz_u = 0;
  int64_t nnzb_kept = 0;                      // blocks of the preconditioner's pattern
  int32_t schedule = 0, nsets = 0;
  std::vector<int32_t> perm, iperm;           // perm[new] = old
  std::vector<int32_t> a_rowptr, l_rowptr, u_rowptr;
  std::vector<int32_t> a_col, l_col, u_col;   // warp-sliced order
  std::vector<int32_t> a_src;                 // per A block (sliced order): caller's block index
  std::vector<int64_t> a_dst;                 // per A block (sliced order): slot in the factor values, -1 if none
  std::vector<int64_t> a_csr_slot;            // per A block in permuted CSR order: slot in the factor values
  std::vector<int32_t> upd_ptr;               // per L block (CSR order of L) into the update lists
  std::vector<int64_t> upd_dst, upd_src;      // slots: A_ij -= L_ik * U_kj
  int64_t nupd = 0;                           // update products (the lists' length)
  // Rows whose every update is A_ii -= L_ik U_ki (no fill-free product lands
  // on an L or U block of the row): the factorisation walks them in one pass
  // with A_ii in registers.  Bit r of fz_mask[s] marks row 32 s + r;
  // a_aux (A's sliced order) holds, for a kept L block (i,k) of such a row,
  // the slot of U_ki, or -1 (no such block, or any other block or row).
  std::vector<uint32_t> fz_mask;
  std::vector<int64_t> a_aux;
  // phases: maximal runs of consecutive (schedule-order) rows none of which
  // reads another row of its run in either sweep; rows [phase_ptr[p],
  // phase_ptr[p+1]) form phase p.  For level and colour orders the phases are
  // exactly the levels and colours.
  std::vector<int32_t> phase_ptr;
  // per 32-row slice, bit r for row 32*slice + r: (x) the row has no U block,
  // so its backward step runs inside the forward sweep; (y) its forward
  // result y is read later (by its own backward step or another row's L).
  std::vector<uint32_t> sl_mask;              // 2 per slice: x, y
  // The BiCGStab products that follow a preconditioner application,
  // v = A p^ with p^ = inv(LU) p.  ILU0 makes (LU)_ij = A_ij on the
  // pattern, so per 32-row slice, bit r for row 32*slice + r:
  // (x) the row has no block left of its diagonal and every block in the
  //     preconditioner: L's row is empty and U's row is A's, so
  //     (A p^)_i = (U p^)_i = p_i;
  // (y) otherwise, U's upper row is A's (every upper block kept, no ILU0
  //     product landed on one): sum_{j>i} A_ij p^_j is the backward
  //     sweep's sum_{j>i} U_ij p^_j, and the product walks only the
  //     diagonal and the blocks left of it.
  // sp_len[i]: the leading blocks of A's row (A's order: the diagonal, then
  // columns ascending) the product walks: 0 (x), 1 + the lower blocks (y),
  // all of them otherwise.
  std::vector<uint32_t> sp_mask;              // 2 per slice: x, y
  std::vector<int32_t> sp_len;
  int64_t nnzb_product = 0;                   // sum of sp_len
  int32_t rows_identity = 0;                  // rows with bit x
  int32_t rows_reuse = 0;                     // rows with bit y
  std::vector<int32_t> sp_tile;               // per 256-row SpMV tile: the blocks the products walk
  int64_t d_off = 0;                          // first value of Dinv inside the factor values
  int64_t lu_vals = 0;                        // total factor values
  int32_t max_row_len = 0;
};

// Validates and analyses the pattern; returns OPM_OK or a pattern error with
// *err_row set to the offending row (caller's numbering).
// part (may be NULL): partition label of every row; blocks joining rows of
// different partitions stay out of the preconditioner (block-Jacobi).
opm_status analyse(int32_t n, const int32_t *rowptr, const int32_t *colidx, const int32_t *part,
                   int32_t schedule, Analysis &an, int32_t *err_row);

// Krylov scalars and control words, one per system, in device memory.
struct alignas(128) DevState {
  double rho, rho_prev, alpha, omega, beta;
  double n0, tol;
  double rhv, ss, ts, tt, rr, rhr;
  double relres;
  double bb;       // ||b||^2 of the setup, when the state is set separately (k_start)
  int32_t status;  // kRunning or an opm_status
  int32_t k;       // current iteration, 1-based
  int32_t iters;
  int32_t maxit;
  int32_t half;    // the last half step met the stopping rule
  int32_t error;   // error detected during the current operation (opm_status) or 0
  int32_t ferror;  // error of the last factorisation, kept until the next one
  int32_t err_row; // smallest permuted row with a singular pivot
  uint32_t red_count;            // last-CTA reduction counter
};

}  // namespace opm
