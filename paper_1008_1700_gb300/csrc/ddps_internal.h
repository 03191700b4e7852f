// Internal declarations of the DDPS library (not part of the ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "ddps.h"

namespace ddps {

// Result of the symbolic phase (host side).  "new" indices are positions in
// the nested-dissection order of each block, offset by the block's first row,
// so a block keeps its row range in both orders.
struct Analysis {
  int64_t n = 0, nnz = 0;
  int32_t p = 0, nsys = 0;
  std::vector<int64_t> block_ptr;      // p+1
  std::vector<int32_t> sys_block_ptr;  // nsys+1
  std::vector<int64_t> sys_row_ptr;    // nsys+1
  std::vector<int32_t> block_sys;      // p

  std::vector<int32_t> perm;   // perm[new] = old (global rows)
  std::vector<int32_t> iperm;  // iperm[old] = new

  // Fronts (supernodes) of all blocks, structure of arrays.
  std::vector<int32_t> f_k, f_m, f_block, f_parent, f_depth, f_cbeg, f_cend;
  std::vector<int64_t> f_row0;   // new index of the first pivot
  std::vector<int64_t> f_arena;  // offset of the m x m column-major front (elements)
  std::vector<int64_t> f_idx;    // offset into idx (m entries: new indices of the front rows)
  std::vector<int64_t> f_upd;    // offset of the r-entry update vector
  std::vector<int64_t> f_rel;    // offset into rel (r entries), -1 for roots
  std::vector<int32_t> idx, rel, children;
  int64_t arena_size = 0, upd_size = 0;
  int32_t nlevels = 0, max_children = 0;
  std::vector<int32_t> level_ptr, level_fronts;  // fronts by depth (0 = roots)
  // extend-add schedule: for parent depth L and child slot s, the child fronts
  std::vector<int32_t> ea_ptr, ea_list;  // ea_ptr[(L * max_children + s)] .. +1

  std::vector<int64_t> amap;  // per stored entry of A: front arena offset, or -1 (entry of R)

  // R~ (kept entries of R), CSR over original rows; columns are reduced indices.
  std::vector<int32_t> rt_rowptr, rt_col, rt_rhscol, rt_rownew;
  std::vector<int64_t> rt_src;  // index of the entry in A's value array

  // Interface set c and the reduced index space.
  std::vector<int64_t> c;            // m global (original) indices, ascending
  std::vector<int64_t> sys_c_ptr;    // nsys+1
  std::vector<int32_t> c_rownew;     // new index of row c[q]
  // Layout of G^ per block: rows [gq0, gq1) of the reduced system, coupling columns.
  std::vector<int64_t> gq0, gq1, gcol_ptr, ghat_off, gld;  // gld: row stride (multiple of 8)
  std::vector<int32_t> gcols;        // reduced indices of the coupling columns (ascending)
  int64_t ghat_entries = 0, max_rhs = 0, max_front = 0, factor_lu_entries = 0;
  double factor_flops = 0, spike_flops = 0;

  // ILU(0) factors (factor_kind ILU0): the blocks keep their own row order
  // (perm is the identity, no fronts); CSR of the diagonal blocks, diagonal
  // positions, and the rows grouped in levels for the L and the U solves
  // (il_lb: level 0 = rows whose U part references no other row).
  bool ilu = false;
  std::vector<int32_t> il_rp, il_col, il_diag, il_row_block;
  std::vector<int32_t> il_lf, il_lf_ptr, il_lb, il_lb_ptr;
};

// Builds the analysis.  Returns an empty string on success, else the error.
std::string analyze(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                    int32_t p, const int64_t* block_ptr, int32_t nsys,
                    const int32_t* sys_block_ptr, const double* values,
                    const ddps_options& opt, Analysis& out);

}  // namespace ddps
