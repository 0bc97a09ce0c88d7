// Internal host-side structures shared by the symbolic analysis, the plan
// builder and the C ABI.  Nothing here is part of the public interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "rsc.h"

namespace rsc {

// In-order labelled binary tree over the columns of one diagonal block
// (Section 4.1, Eq. "ldjLabel").  Arrays are indexed by label 1..nblocks
// (index 0 unused).  Leaf s covers columns [lo, hi); internal s is the block
// with rows [mid, hi) and columns [lo, mid).  Ranges are local to the supernode.
struct BlockTree {
    int nblocks = 0;
    int root = 0;
    std::vector<uint8_t> leaf;
    std::vector<int32_t> lo, mid, hi, left, right, parent;
};

struct Symbolic {
    int64_t n = 0;
    int dof = 1;
    int M = 0;                              // supernodes
    std::vector<int32_t> perm, iperm;       // perm[new] = old
    int ncomp = 1;                          // connected components of the node graph
    bool graph_ordering = false;            // graph nested dissection (else lattice bisection)
    std::vector<double> node_pos;           // [n / dof * 3] positions the ordering used
    std::vector<int32_t> comp_of;           // [n / dof] component of each node (original order)
    std::vector<int64_t> sn_ptr;            // [M+1] column boundaries
    std::vector<int32_t> snode_of;          // [n] supernode of each (new) column
    std::vector<uint8_t> kind;              // 0 leaf, 1 separator
    std::vector<int64_t> rows_ptr;          // [M+1]
    std::vector<int32_t> rows;              // R_j, sorted new row indices after C_j
    std::vector<int32_t> parent, level;
    int nlevels = 0;
    std::vector<std::vector<int32_t>> level_nodes;
    std::vector<BlockTree> tree;            // per supernode, nblocks == 0 if none
    // D_j: for each j the descendants k with R_k meeting C_j (ascending k); rows
    // p0..p1-1 of R_k fall in C_j (a contiguous run), rows p1.. fall in R_j.
    std::vector<int64_t> desc_ptr;
    std::vector<int32_t> desc_k, desc_p0, desc_p1;
    // Permuted lower triangle of A by column: entries (li, c) with li >= c and
    // the index lsrc into the caller's value array.
    std::vector<int64_t> lp;
    std::vector<int32_t> li;
    std::vector<int64_t> lsrc;

    int ncols(int j) const { return (int)(sn_ptr[j + 1] - sn_ptr[j]); }
    int nrows(int j) const { return (int)(rows_ptr[j + 1] - rows_ptr[j]); }
    const int32_t* R(int j) const { return rows.data() + rows_ptr[j]; }
};

// Graph ordering (graph_order.cpp): node graph of A's pattern (CSR, sorted, no self
// loops), spectral positions per component (nodes x 3), graph nested dissection of one
// component (parts: 0 leaf / 1 separator, in postorder).
void node_graph(int64_t n, const int64_t* rp, const int32_t* ci, int dof, std::vector<int64_t>& ptr,
                std::vector<int32_t>& idx);
void spectral_positions(const std::vector<int64_t>& ptr, const std::vector<int32_t>& idx,
                        const std::vector<std::vector<int32_t>>& comps, std::vector<double>& X);
void graph_nested_dissection(const std::vector<int64_t>& ptr, const std::vector<int32_t>& idx, const double* X,
                             int leaf_size, std::vector<int32_t>& ids,
                             std::vector<std::pair<uint8_t, std::vector<int32_t>>>& parts);

// Ordering + symbolic analysis; returns an empty string on success, else the reason.
std::string analyze_symbolic(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                             const double* coords, const rsc_options& opts, Symbolic& S);

}  // namespace rsc
