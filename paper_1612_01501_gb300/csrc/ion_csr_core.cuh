// ion_csr_core.cuh -- the per-row CSR gap-junction sum shared by the single-network
// kernel (ion_csr.cu) and the batched kernel (ion_batch.cu).
#pragma once
#include <cstdint>

#include "ion_kernels.cuh"

namespace ion {

__device__ __forceinline__ float gj_edge(float vi, float vj, float w) {
    const float du = (vi - vj) * GJ_SCALE;
    return w * fmaf(0.8f, ex2_approx(-du * du), 0.2f) * du;
}
// The junction term of one edge, in the same scaled units: LIN selects the linear
// junction of the SGJ use case (Sec. 2.3.2), w (V_i - V_j) s, else the term above.
template <bool LIN>
__device__ __forceinline__ float jn_edge(float vi, float vj, float w) {
    return LIN ? w * ((vi - vj) * GJ_SCALE) : gj_edge(vi, vj, w);
}

// Sum of one row's edges [e0, e1) handled by lane li of an SW-lane group.  VEC: the index
// and weight arrays are 16-byte aligned, so the body of the row is read four edges per
// lane with one 16-byte load each (a head of up to three edges and a tail are read one
// by one).  Four V_dend gathers are in flight per lane per iteration.
template <int SW, bool VEC, bool HAS_W>
__device__ __forceinline__ float csr_row_sum(const float *__restrict__ vcur, const int32_t *__restrict__ col,
                                             const float *__restrict__ w, int e0, int e1, float vi, int li) {
    float acc = 0.0f;
    if (VEC) {
        const int ea = min(e1, (e0 + 3) & ~3);                 // first 16-byte aligned edge
        const int eb = ea + ((e1 - ea) & ~3);                   // end of the aligned body
        for (int e = e0 + li; e < ea; e += SW) acc += gj_edge(vi, __ldg(vcur + __ldg(col + e)), HAS_W ? __ldg(w + e) : 1.0f);
        for (int e = ea + 4 * li; e < eb; e += 4 * SW) {
            const int4 j = __ldg(reinterpret_cast<const int4 *>(col + e));
            float4 ww = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
            if (HAS_W) ww = __ldg(reinterpret_cast<const float4 *>(w + e));
            const float v0 = __ldg(vcur + j.x), v1 = __ldg(vcur + j.y), v2 = __ldg(vcur + j.z), v3 = __ldg(vcur + j.w);
            acc += (gj_edge(vi, v0, ww.x) + gj_edge(vi, v1, ww.y)) + (gj_edge(vi, v2, ww.z) + gj_edge(vi, v3, ww.w));
        }
        for (int e = eb + li; e < e1; e += SW) acc += gj_edge(vi, __ldg(vcur + __ldg(col + e)), HAS_W ? __ldg(w + e) : 1.0f);
    } else {
        int e = e0 + li;
        for (; e + 3 * SW < e1; e += 4 * SW) {
            const int j0 = __ldg(col + e), j1 = __ldg(col + e + SW), j2 = __ldg(col + e + 2 * SW), j3 = __ldg(col + e + 3 * SW);
            const float w0 = HAS_W ? __ldg(w + e) : 1.0f, w1 = HAS_W ? __ldg(w + e + SW) : 1.0f;
            const float w2 = HAS_W ? __ldg(w + e + 2 * SW) : 1.0f, w3 = HAS_W ? __ldg(w + e + 3 * SW) : 1.0f;
            const float v0 = __ldg(vcur + j0), v1 = __ldg(vcur + j1), v2 = __ldg(vcur + j2), v3 = __ldg(vcur + j3);
            acc += (gj_edge(vi, v0, w0) + gj_edge(vi, v1, w1)) + (gj_edge(vi, v2, w2) + gj_edge(vi, v3, w3));
        }
        for (; e < e1; e += SW) acc += gj_edge(vi, __ldg(vcur + __ldg(col + e)), HAS_W ? __ldg(w + e) : 1.0f);
    }
    return acc;
}

// Sum of one row's edges [e0, e1) whose columns all lie in the shared-memory chunk that
// starts at global column c0 (vs holds V_dend[c0 ...]).  Same lane layout as csr_row_sum.
template <int SW, bool VEC, bool HAS_W>
__device__ __forceinline__ float csr_row_sum_smem(const float *vs, int c0, const int32_t *__restrict__ col,
                                                  const float *__restrict__ w, int e0, int e1, float vi, int li) {
    float acc = 0.0f;
    if (VEC) {
        const int ea = min(e1, (e0 + 3) & ~3);
        const int eb = ea + ((e1 - ea) & ~3);
        for (int e = e0 + li; e < ea; e += SW) acc += gj_edge(vi, vs[__ldg(col + e) - c0], HAS_W ? __ldg(w + e) : 1.0f);
        for (int e = ea + 4 * li; e < eb; e += 4 * SW) {
            const int4 j = __ldcs(reinterpret_cast<const int4 *>(col + e));     // streamed once per step
            float4 ww = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
            if (HAS_W) ww = __ldcs(reinterpret_cast<const float4 *>(w + e));
            const float v0 = vs[j.x - c0], v1 = vs[j.y - c0], v2 = vs[j.z - c0], v3 = vs[j.w - c0];
            acc += (gj_edge(vi, v0, ww.x) + gj_edge(vi, v1, ww.y)) + (gj_edge(vi, v2, ww.z) + gj_edge(vi, v3, ww.w));
        }
        for (int e = eb + li; e < e1; e += SW) acc += gj_edge(vi, vs[__ldg(col + e) - c0], HAS_W ? __ldg(w + e) : 1.0f);
    } else {
        for (int e = e0 + li; e < e1; e += SW) acc += gj_edge(vi, vs[__ldg(col + e) - c0], HAS_W ? __ldg(w + e) : 1.0f);
    }
    return acc;
}

// Two edges of row i at once through packed f32x2 arithmetic (the same terms as gj_edge):
// dV = V_i - V_j (an FFMA2 with -1: the same bits as a subtraction), du = dV s, then
// acc += w (0.8 2^{-du^2} + 0.2) du, the last product fused into the accumulation.
// LIN: the linear junction, acc += w du (jn_edge).
template <bool HAS_W, bool LIN = false>
__device__ __forceinline__ float2 gj_edge2(float2 vi2, float2 vj2, float2 w2, float2 acc) {
    const float2 d = __ffma2_rn(vj2, make_float2(-1.0f, -1.0f), vi2);
    const float2 du = __fmul2_rn(d, make_float2(GJ_SCALE, GJ_SCALE));
    if (LIN) return HAS_W ? __ffma2_rn(w2, du, acc) : __fadd2_rn(du, acc);
    const float2 q = __fmul2_rn(du, du);
    const float2 e = make_float2(ex2_approx(-q.x), ex2_approx(-q.y));
    float2 f = __ffma2_rn(e, make_float2(0.8f, 0.8f), make_float2(0.2f, 0.2f));
    if (HAS_W) f = __fmul2_rn(f, w2);
    return __ffma2_rn(f, du, acc);
}

// Eight edges of a 16-byte group of 16-bit columns (and their weights), two at a time.
template <bool HAS_W, bool LIN = false, class VJ>
__device__ __forceinline__ float csr_group16(uint4 q, float4 wa, float4 wb, float vi, VJ vj) {
    const float2 vi2 = make_float2(vi, vi);
    float2 acc = make_float2(0.0f, 0.0f);
    acc = gj_edge2<HAS_W, LIN>(vi2, make_float2(vj(q.x & 0xFFFFu), vj(q.x >> 16)), make_float2(wa.x, wa.y), acc);
    acc = gj_edge2<HAS_W, LIN>(vi2, make_float2(vj(q.y & 0xFFFFu), vj(q.y >> 16)), make_float2(wa.z, wa.w), acc);
    acc = gj_edge2<HAS_W, LIN>(vi2, make_float2(vj(q.z & 0xFFFFu), vj(q.z >> 16)), make_float2(wb.x, wb.y), acc);
    acc = gj_edge2<HAS_W, LIN>(vi2, make_float2(vj(q.w & 0xFFFFu), vj(q.w >> 16)), make_float2(wb.z, wb.w), acc);
    return acc.x + acc.y;
}
template <bool HAS_W, bool LD_STREAM>
__device__ __forceinline__ void csr_load16(const uint16_t *__restrict__ col16, const float *__restrict__ w, int e,
                                           uint4 &q, float4 &wa, float4 &wb) {
    q = LD_STREAM ? __ldcs(reinterpret_cast<const uint4 *>(col16 + e)) : __ldg(reinterpret_cast<const uint4 *>(col16 + e));
    wa = wb = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
    if (HAS_W) {
        wa = LD_STREAM ? __ldcs(reinterpret_cast<const float4 *>(w + e)) : __ldg(reinterpret_cast<const float4 *>(w + e));
        wb = LD_STREAM ? __ldcs(reinterpret_cast<const float4 *>(w + e + 4))
                       : __ldg(reinterpret_cast<const float4 *>(w + e + 4));
    }
}

template <bool LD_STREAM>
__device__ __forceinline__ uint32_t csr_ld16(const uint16_t *__restrict__ col16, int e) {
    return LD_STREAM ? (uint32_t)__ldcs(col16 + e) : (uint32_t)__ldg(col16 + e);
}

// 16-bit column indices: col16[e] holds the low 16 bits of column e (exact when the
// network has at most 65 536 cells; chunk-relative below).  A row is read as an unaligned
// head (< 8 edges), a body of 16-byte groups of eight edges and a tail (< 8 edges).  With
// eight or more lanes per row the head and tail take one load per lane, and each lane
// issues them together with its first two body groups before using any, so a row costs
// one memory latency rather than one per part (rows of up to 16 x SW body edges are then
// done in one round).  vj maps a 16-bit index to V_dend of that column.  LD_STREAM: the
// indices are read once per step (evict-first), else through the read-only cache.  LIN:
// linear junctions (jn_edge).  ALIGNED: e0 and e1 are multiples of 8 (the padded layout),
// so the row is all body.
template <int SW, bool HAS_W, bool LD_STREAM, bool LIN = false, bool ALIGNED = false, class VJ>
__device__ __forceinline__ float csr_row_sum16(const uint16_t *__restrict__ col16, const float *__restrict__ w,
                                               int e0, int e1, float vi, int li, VJ vj) {
    float acc = 0.0f;
    const int ea = ALIGNED ? e0 : min(e1, (e0 + 7) & ~7);   // first 16-byte aligned edge
    const int eb = ALIGNED ? e1 : ea + ((e1 - ea) & ~7);     // end of the aligned body
    int e = ea + 8 * li;
    if (SW >= 8) {
        const int eh = e0 + li, et = eb + li;
        const bool hh = !ALIGNED && eh < ea, ht = !ALIGNED && et < e1;
        const uint32_t jh = hh ? csr_ld16<LD_STREAM>(col16, eh) : 0u;
        const uint32_t jt = ht ? csr_ld16<LD_STREAM>(col16, et) : 0u;
        const float wh = (HAS_W && hh) ? __ldg(w + eh) : 1.0f, wt = (HAS_W && ht) ? __ldg(w + et) : 1.0f;
        const bool g0 = e < eb, g1 = e + 8 * SW < eb;
        uint4 q0 = make_uint4(0u, 0u, 0u, 0u), q1 = q0;
        float4 a0 = make_float4(1.0f, 1.0f, 1.0f, 1.0f), b0 = a0, a1 = a0, b1 = a0;
        if (g0) csr_load16<HAS_W, LD_STREAM>(col16, w, e, q0, a0, b0);
        if (g1) csr_load16<HAS_W, LD_STREAM>(col16, w, e + 8 * SW, q1, a1, b1);
        if (hh) acc += jn_edge<LIN>(vi, vj(jh), wh);
        if (ht) acc += jn_edge<LIN>(vi, vj(jt), wt);
        if (g0) acc += csr_group16<HAS_W, LIN>(q0, a0, b0, vi, vj);
        if (g1) acc += csr_group16<HAS_W, LIN>(q1, a1, b1, vi, vj);
        e += 16 * SW;
    } else if (!ALIGNED) {
        for (int eh = e0 + li; eh < ea; eh += SW) acc += jn_edge<LIN>(vi, vj(csr_ld16<LD_STREAM>(col16, eh)), HAS_W ? __ldg(w + eh) : 1.0f);
    }
    if (!HAS_W) {   // long rows: four groups (64 B of indices per lane) in flight per round
        for (; e + 24 * SW < eb; e += 32 * SW) {
            uint4 q0, q1, q2, q3;
            float4 u0, u1;
            csr_load16<false, LD_STREAM>(col16, w, e, q0, u0, u1);
            csr_load16<false, LD_STREAM>(col16, w, e + 8 * SW, q1, u0, u1);
            csr_load16<false, LD_STREAM>(col16, w, e + 16 * SW, q2, u0, u1);
            csr_load16<false, LD_STREAM>(col16, w, e + 24 * SW, q3, u0, u1);
            acc += (csr_group16<false, LIN>(q0, u0, u1, vi, vj) + csr_group16<false, LIN>(q1, u0, u1, vi, vj)) +
                   (csr_group16<false, LIN>(q2, u0, u1, vi, vj) + csr_group16<false, LIN>(q3, u0, u1, vi, vj));
        }
    }
    for (; e + 8 * SW < eb; e += 16 * SW) {                 // further rounds: two groups in flight
        uint4 q0, q1;
        float4 a0, b0, a1, b1;
        csr_load16<HAS_W, LD_STREAM>(col16, w, e, q0, a0, b0);
        csr_load16<HAS_W, LD_STREAM>(col16, w, e + 8 * SW, q1, a1, b1);
        acc += csr_group16<HAS_W, LIN>(q0, a0, b0, vi, vj) + csr_group16<HAS_W, LIN>(q1, a1, b1, vi, vj);
    }
    if (e < eb) {
        uint4 q;
        float4 a, b;
        csr_load16<HAS_W, LD_STREAM>(col16, w, e, q, a, b);
        acc += csr_group16<HAS_W, LIN>(q, a, b, vi, vj);
    }
    if (SW < 8 && !ALIGNED)
        for (int et = eb + li; et < e1; et += SW) acc += jn_edge<LIN>(vi, vj(csr_ld16<LD_STREAM>(col16, et)), HAS_W ? __ldg(w + et) : 1.0f);
    return acc;
}

// V_dend of a full 16-bit column index, from global memory (networks of <= 65 536 cells)
struct VjGlobal {
    const float *v;
    __device__ __forceinline__ float operator()(uint32_t j) const { return __ldg(v + j); }
};
// The same through L2 only (ld.global.cg): for data other CTAs of a persistent launch wrote
// earlier in the same launch, which the non-coherent read-only and L1 paths may hold stale
struct VjGlobalCG {
    const float *v;
    __device__ __forceinline__ float operator()(uint32_t j) const { return __ldcg(v + j); }
};
// V_dend of a column of the shared-memory chunk starting at c0 (a multiple of 32 768):
// the column lies in [c0, c0 + 32 768), so its low 15 bits are its offset in the chunk
// (j holds the column's low 16 bits, possibly with other bits above them)
static_assert(CSR_CHUNK == 32768, "chunk-relative columns are the low 15 bits");
struct VjChunk {
    const float *vs;
    __device__ __forceinline__ float operator()(uint32_t j) const { return vs[j & 0x7FFFu]; }
};
// The padded layout's columns are chunk-relative already; the padding entries index slots
// past the chunk that hold each row's own V_dend
struct VjPadded {
    const float *vs;
    __device__ __forceinline__ float operator()(uint32_t j) const { return vs[j]; }
};

}  // namespace ion
