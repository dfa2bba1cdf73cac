// tc_split.cuh -- limb operands of the tensor-core SYRDK (syrdk_tc.cu).
//
// A residue in balanced form (-p/2, p/2] is split into signed digits that
// bf16 holds exactly; split_write() stores one row's digits for eight
// consecutive K columns in the pre-tiled core-matrix layout that the SYRDK
// kernel copies stage by stage: the A operand (digits of G D, L_A digits of
// base 2^ash) in 128-row blocks, the B operand (base-256 digits of the
// pre-scaled copies beta^u G, u < L_A) in bn-row blocks with the L_B digit
// planes stacked along N.  Used by the panel update's split kernel and by the
// fused TRSS block step (trss.cu).
#pragma once

#include <cuda_bf16.h>

#include "ldlt_internal.cuh"

constexpr int TC_BM = 128;  // rows per A-operand block (the SYRDK tile's M)

__device__ __forceinline__ int32_t balanced(uint32_t x, uint32_t p)
{
    return x > (p >> 1) ? (int32_t)((int64_t)x - (int64_t)p) : (int32_t)x;
}

// digit u of the balanced base-2^sh expansion (top digit takes the rest)
__device__ __forceinline__ void digits(int32_t x, int L, int sh, int32_t *d)
{
    const int32_t half = 1 << (sh - 1), mask = (1 << sh) - 1;
    for (int u = 0; u < L - 1; ++u) {
        int32_t lo = ((x + half) & mask) - half;
        d[u] = lo;
        x = (x - lo) >> sh;
    }
    d[L - 1] = x;
}

__device__ __forceinline__ uint4 pack8(const int32_t *v)
{
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        __nv_bfloat16 lo = __float2bfloat16_rn((float)v[2 * h]);
        __nv_bfloat16 hi = __float2bfloat16_rn((float)v[2 * h + 1]);
        w[h] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

struct SplitArgs {
    const uint32_t *LpC;
    int64_t ldL;
    const int *sigma;
    int la, ash, lb, bn, nprime;  // A: la digits of base 2^ash
    const LoopState *ls;          // with out: m_next rows, np columns
    const PanelOut *out;
    const uint32_t *S;            // np = 0: Snext = S[sigma, sigma]
    int64_t ldS;
    uint32_t *Snext;
    FieldP f;
    uint32_t wbase[4];  // beta^u mod p
    __nv_bfloat16 *Aop, *Bop;
};

// Write the limb operands of row i, columns k0 .. k0+7: the digits of GD
// (A operand) and of the pre-scaled copies of G (B operand), in the pre-tiled
// core-matrix layouts the SYRDK kernel copies stage by stage.
__device__ __forceinline__ void split_write(const SplitArgs &a, int i, int k0, int kpad, int kprime, int rows,
                                            const int32_t (&gd_bal)[8], const uint32_t (&gk)[8])
{
    const FieldP f = a.f;
    const int LA = a.la, LB = a.lb;
    int32_t gb[8];
    // A operand: digit u of GD at K' column u*kpad + k
    const int I = i / TC_BM, ri = i % TC_BM;
    const int J = i / a.bn, rj = i % a.bn;
    int32_t dg[8][4];
#pragma unroll
    for (int e = 0; e < 8; ++e) digits(gd_bal[e], LA, a.ash, dg[e]);
    for (int u = 0; u < LA; ++u) {
        int32_t v8[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v8[e] = dg[e][u];
        const int kk = u * kpad + k0;
        const int64_t off = (int64_t)I * TC_BM * kprime + (int64_t)(kk / 8) * (TC_BM * 8) + ri * 8;
        *(uint4 *)(a.Aop + off) = pack8(v8);
    }
    // B operand: base-256 digit v of b~_u = balanced(beta^u g mod p), rows v*bn + rj
    if (i < ((rows + a.bn - 1) / a.bn) * a.bn) {
        for (int u = 0; u < LA; ++u) {
            int32_t db[8][4];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                gb[e] = balanced(fp_mul(a.wbase[u], gk[e], f), f.p);
                digits(gb[e], LB, 8, db[e]);
            }
            const int kk = u * kpad + k0;
            for (int v = 0; v < LB; ++v) {
                int32_t v8[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) v8[e] = db[e][v];
                const int64_t off = (int64_t)J * a.nprime * kprime + (int64_t)(kk / 8) * (a.nprime * 8) +
                                    (int64_t)(v * a.bn + rj) * 8;
                *(uint4 *)(a.Bop + off) = pack8(v8);
            }
        }
    }
}


// Arguments of split_write for an update whose operands are formed by the
// caller (no panel record, no row map): the field, the digit counts and bases
// of a prime, and the two operand buffers.  Host side (syrdk_tc.cu).
SplitArgs tc_split_args(FieldP f, int limbs, void *Aop, void *Bop);
