// ion_bank.cu -- host-side edge order for the shared-memory gathers of the staged CSR
// kernel (no device code).
//
// The staged kernel sums a row's edges whose columns fall in one V_dend chunk of
// `chunk` cells (a multiple of 32), gathering V_dend from shared memory.  With
// `lanes` lanes per row it reads the 16-byte-aligned body of the row's segment as groups
// of eight 16-bit columns: lane l takes groups l, l + lanes, l + 2 lanes, ..., and one
// gather instruction reads position k (0..7) of the groups of one round, i.e. the edges
//   body_start + 8 (r lanes + l) + k,   l = 0 .. lanes - 1,
// whose shared-memory banks are their columns mod 32.  For a random graph those banks
// collide (about four wavefronts per 32-lane gather).  The sum of a row does not depend on
// the order of its edges beyond rounding, so the edges of each body can be placed such
// that every such gather set takes distinct banks where the row allows it: sets are
// filled one at a time, each from the banks with the most edges left (ties to the lower
// bank), which keeps the remaining banks balanced.  Heads and tails (the unaligned ends
// of a segment, read one edge per lane) keep their order, and no edge leaves its segment,
// so every column stays in the chunk the kernel has staged for that position.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ion.h"
#include "ion_sim.h"

namespace {

struct BankBuckets {
    std::vector<int32_t> edges[32];
    size_t next[32];
    void reset() {
        for (int b = 0; b < 32; ++b) {
            edges[b].clear();
            next[b] = 0;
        }
    }
    size_t left(int b) const { return edges[b].size() - next[b]; }
};

// Place the body [ea, eb) of one segment (eb - ea a multiple of 8) into perm.
void order_body(const int32_t *col, int32_t ea, int32_t eb, int lanes, BankBuckets &B, int32_t *perm) {
    const int G = (eb - ea) / 8;
    B.reset();
    for (int32_t e = ea; e < eb; ++e) B.edges[col[e] & 31].push_back(e);
    int order[32];
    for (int r = 0; r * lanes < G; ++r) {
        const int m = std::min(lanes, G - r * lanes);   // groups (lanes) of this round
        for (int k = 0; k < 8; ++k) {
            for (int b = 0; b < 32; ++b) order[b] = b;
            std::stable_sort(order, order + 32, [&](int x, int y) { return B.left(x) > B.left(y); });
            int placed = 0;
            for (int q = 0; q < 32 && placed < m; ++q) {   // one edge from each of the fullest banks
                const int b = order[q];
                if (B.left(b) == 0) break;
                perm[ea + 8 * (r * lanes + placed) + k] = B.edges[b][B.next[b]++];
                ++placed;
            }
            while (placed < m) {   // fewer non-empty banks than lanes: collisions are unavoidable
                int best = -1;
                for (int b = 0; b < 32; ++b)
                    if (B.left(b) > 0 && (best < 0 || B.left(b) > B.left(best))) best = b;
                perm[ea + 8 * (r * lanes + placed) + k] = B.edges[best][B.next[best]++];
                ++placed;
            }
        }
    }
}

}  // namespace

extern "C" ion_status ion_csr_bank_order(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t chunk,
                                         int32_t lanes_per_row, int32_t *perm) {
    if (n < 1 || !row_ptr || !perm || chunk < 32 || chunk % 32 != 0 ||
        (lanes_per_row != 8 && lanes_per_row != 16 && lanes_per_row != 32))
        return ION_ERR_INVALID_ARG;
    if (row_ptr[0] != 0) return ION_ERR_BAD_CSR;
    for (int32_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return ION_ERR_BAD_CSR;
    const int32_t nnz = row_ptr[n];
    if (nnz > 0 && !col_idx) return ION_ERR_INVALID_ARG;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = row_ptr[i] + 1; e < row_ptr[i + 1]; ++e)
            if (col_idx[e] <= col_idx[e - 1]) return ION_ERR_BAD_CSR;   // ascending per row
    for (int32_t e = 0; e < nnz; ++e) perm[e] = e;
    BankBuckets B;
    for (int32_t i = 0; i < n; ++i) {
        int32_t s0 = row_ptr[i];
        const int32_t end = row_ptr[i + 1];
        while (s0 < end) {   // one segment per chunk of columns
            const int64_t c_end = ((int64_t)col_idx[s0] / chunk + 1) * chunk;
            int32_t s1 = s0;
            while (s1 < end && col_idx[s1] < c_end) ++s1;
            const int32_t ea = std::min(s1, (s0 + 7) & ~7);   // first 16-byte aligned edge
            const int32_t eb = ea + ((s1 - ea) & ~7);          // end of the aligned body
            if (eb > ea) order_body(col_idx, ea, eb, lanes_per_row, B, perm);
            s0 = s1;
        }
    }
    return ION_OK;
}

// The 16-bit columns of a host CSR (sorted rows) in bank order for the lane count the
// staged kernel will use (the degree-based choice of ion_setup_csr_staging), padded with
// zeros to whole 16-byte groups.  Every position is checked to hold an edge of its own
// row whose column lies in the same chunk as the edge the sorted order puts there (so the
// kernel's chunk-relative index stays inside the staged chunk).  Returns false, leaving
// `out` unused, when the lane count has no grouped body (fewer than 8 lanes), the order
// cannot be built, or the check fails.
bool ion_csr_bank_col16(int32_t n, int32_t n_pad, const int32_t *row_ptr, const int32_t *col,
                        std::vector<uint16_t> &out) {
    const int64_t nnz = row_ptr[n];
    if (nnz <= 0) return false;
    const int n_chunks = (n_pad + ion::CSR_CHUNK - 1) / ion::CSR_CHUNK;
    int sw = 0, rows_unused = 0;
    ion_choose_csr_shape((double)nnz / n / n_chunks, &sw, &rows_unused);
    if (sw < 8) return false;
    std::vector<int32_t> perm((size_t)nnz);
    if (ion_csr_bank_order(n, row_ptr, col, ion::CSR_CHUNK, sw, perm.data()) != ION_OK) return false;
    std::vector<uint8_t> seen((size_t)nnz, 0);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int32_t p = perm[(size_t)e];
            if (p < row_ptr[i] || p >= row_ptr[i + 1] || seen[(size_t)p]) return false;
            if (col[p] / ion::CSR_CHUNK != col[e] / ion::CSR_CHUNK) return false;
            seen[(size_t)p] = 1;
        }
    out.assign((size_t)((nnz + 7) & ~(int64_t)7), 0);
    for (int64_t e = 0; e < nnz; ++e) out[(size_t)e] = (uint16_t)(col[perm[(size_t)e]] & 0xFFFF);
    return true;
}
