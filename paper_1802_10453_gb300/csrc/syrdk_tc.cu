// syrdk_tc.cu -- tensor-core form of the level-3 update of Algorithm 2:
//   Z = C - G D G^T   (SYRDK, Section 3), lower triangle, rows compacted.
//
// Exact modular products on bf16 tensor cores.  Every residue is written in
// balanced form (-p/2, p/2] and split into signed digits, small integers that
// bf16 holds exactly (|d| <= 256).  The A side (G D) uses L_A digits of base
// beta (256, or 512 when that needs fewer digits: p in (2^24, 2^26]), digits
// in [-beta/2, beta/2]; the B side uses L_B base-256 digits in [-128, 128].
// With the pre-scaled copies of the B operand
//   b~_u = balanced(beta^u * g mod p),   u < L_A,
// the product sum_k gd_k g_k is congruent mod p to
//   sum_v 256^v * acc_v,   acc_v = sum_u sum_k digit_u(gd_k) * digit_v(b~_u,k),
// so each acc_v is ONE matrix product of inner dimension K' = L_A*K: the A
// operand is [digit_0(GD) | ... | digit_{L_A-1}(GD)] and the B operand for
// acc_v is [digit_v(b~_0) | ... | digit_v(b~_{L_A-1})].  The L_B B operands are
// stacked along N, so a single tcgen05.mma (kind::f16, M = 128, N = L_B*BN) per
// K-step produces all acc_v for a 128 x BN output tile.  The FP32 accumulation
// is exact: |acc_v| <= K' * (beta/2) * 128 <= 3 * 128 * 2^15 < 2^24 with base
// 512 (L_A <= 3) and <= 4 * 128 * 2^14 = 2^23 with base 256.  The epilogue
// reads the L_B accumulators from tensor memory, forms sum_v 256^v acc_v in
// 64-bit integers, reduces once mod p and subtracts from the old Schur entry.
//
// Kernel structure (one CTA per SM, persistent over the lower-triangle tiles):
//   warp 0      bulk-copy producer (cp.async.bulk, mbarrier complete_tx)
//   warp 1      TMEM allocator and MMA issuer (tcgen05.mma, tcgen05.commit)
//   warps 2..17 epilogue, two groups of eight warps taking alternate tiles
//               (tcgen05.ld -> recombine -> mod p -> subtract from the old
//               values gathered into shared memory -> vector stores)
// Operands are pre-tiled in HBM by split_tc_kernel so every pipeline stage is
// one contiguous bulk copy that lands in the no-swizzle K-major "core matrix"
// layout the tensor core reads (8 rows x 16 bytes per core matrix).
#include <cuda_bf16.h>

#include "ldlt_internal.cuh"
#include "tc_split.cuh"

#define LDLT_ERR_TIMEOUT_CODE (-6)

namespace {

constexpr int BM = TC_BM;          // rows per output tile (MMA M)
constexpr int BN = 64;             // output columns per tile (N' = L * BN <= 256)
constexpr int CLD = BN + 4;        // row stride (words) of a prefetched tile of old values
constexpr int KST = 64;            // K' elements per pipeline stage

constexpr int STAGE_A = BM * KST * 2;        // 16 KB
constexpr int STAGE_B_MAX = 256 * KST * 2;   // 32 KB
constexpr int STAGE_BYTES = STAGE_A + STAGE_B_MAX;
constexpr int EPI_WARPS = 16;      // two groups of eight warps (two per TMEM lane quarter)
constexpr int GROUP_THREADS = EPI_WARPS / 2 * 32;
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int TC_THREADS = 64 + EPI_THREADS;
constexpr int NST = 3;             // pipeline stages

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ int64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (int64_t)t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait used only to drain in-flight work before the CTA exits: ignores the
// abort flag and allows at least one second.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity, int64_t budget)
{
    const int64_t lim = budget > 1000000000LL ? budget : 1000000000LL;
    const int64_t t0 = gtime();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (gtime() - t0 > lim) return false;
    }
}

// Bounded wait: false when the budget ran out or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int64_t budget,
                                          volatile int *abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    int64_t t0 = 0;
    for (unsigned n = 1;; ++n) {
        if (mbar_try(bar, parity)) return true;
        if ((n & 255u) == 0) {  // the abort flag and the clock are read once every 256 tries
            if (*abort_flag) return false;
            const int64_t t = gtime();
            if (t0 == 0) t0 = t;
            else if (t - t0 > budget) return false;
        }
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05), no swizzle, K-major:
// start >> 4 in [0,14), LBO >> 4 in [16,30), SBO >> 4 in [32,46), version 1 in
// [46,48), base offset 0, layout type 0 (no swizzle) in [61,64).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A bf16 (7-9 = 1),
// B bf16 (10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at 17, M >> 4 at 24.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------------------
// tile enumeration: lower-triangle tiles (I, J), 128-row blocks, BN-col blocks
// ---------------------------------------------------------------------------
struct TileMap {
    int nI, c, nfull, nlast;  // c = BM / BN; nfull = tiles in the first nI-1 row blocks
};

__device__ __forceinline__ void tile_of(const TileMap &tm, int t, int &I, int &J)
{
    if (t < tm.nfull) {
        // c * I (I + 1) / 2 <= t < c (I + 1)(I + 2) / 2
        int i = (int)((sqrtf(8.0f * (float)t / (float)tm.c + 1.0f) - 1.0f) * 0.5f);
        while (tm.c * (i + 1) * (i + 2) / 2 <= t) ++i;
        while (i > 0 && tm.c * i * (i + 1) / 2 > t) --i;
        I = i;
        J = t - tm.c * i * (i + 1) / 2;
    } else {
        I = tm.nI - 1;
        J = t - tm.nfull;
    }
}

struct TcArgs {
    const uint32_t *S;
    int64_t ldS;
    const int *sigma;
    const LoopState *ls;            // with out: m_next rows, K = np (padded to kpad)
    const PanelOut *out;
    const __nv_bfloat16 *Aop;
    const __nv_bfloat16 *Bop;
    int limbs, bn, nprime, la;      // N' = L_B * bn (limbs = L_B), K' = L_A * kpad (la = L_A)
    FieldP f;
    uint64_t bias;                  // multiple of p above 2^50
    uint32_t *Snext;
    int64_t budget_ns;
    int32_t *status;
    int test_drop;                  // LDLT_TEST_DROP_UPDATE_COPIES: producer stops after one stage
    int upper;                      // 1: output (i, j), j <= i, lives at S[j][i] (the upper triangle;
                                    // S and Snext the same block, sigma the identity)
    int nst;
};

__global__ void __launch_bounds__(TC_THREADS, 1) syrdk_tc_kernel(const TcArgs args)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *stages = smem;
    uint32_t *cold = (uint32_t *)(smem + NST * STAGE_BYTES);  // [2 groups][BM][CLD]: old Schur values
    uint64_t *bars = (uint64_t *)(smem + NST * STAGE_BYTES + 2 * BM * CLD * 4);
    // bars[0..NST) full, [NST..2NST) empty, [2NST, 2NST+2) tmem full,
    // [2NST+2, 2NST+4) tmem empty, [2NST+4] drain
    uint32_t *tmem_holder = (uint32_t *)(bars + 2 * NST + 5);
    volatile int *abort_flag = (volatile int *)(tmem_holder + 1);

    // sizes of this panel's update (written by the kernels before this one);
    // a CTA without a tile returns before it takes tensor memory
    if (!step_live(args.ls, args.out)) return;
    const int m_next = args.out->m_next, npiv = args.out->np;
    if (m_next == 0 || npiv == 0) return;
    const int kprime = args.la * ((npiv + 63) / 64 * 64);
    TileMap tm;
    tm.nI = (m_next + BM - 1) / BM;
    tm.c = BM / args.bn;
    tm.nfull = tm.c * (tm.nI - 1) * tm.nI / 2;
    tm.nlast = (m_next + args.bn - 1) / args.bn;
    const int ntiles = tm.nfull + tm.nlast;
    if ((int)blockIdx.x >= ntiles) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = kprime / KST;
    const int np_ = args.nprime;
    const uint32_t stageB_bytes = (uint32_t)np_ * KST * 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[NST + s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bars[2 * NST + b]), 1);
            mbar_init(smem_u32(&bars[2 * NST + 2 + b]), EPI_THREADS / 2);
        }
        mbar_init(smem_u32(&bars[2 * NST + 4]), 1);  // drain barrier
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_holder)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    if (warp == 0) {
        // ---------------- producer ----------------
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int I, J;
                tile_of(tm, t, I, J);
                const __nv_bfloat16 *ablk = args.Aop + (int64_t)I * BM * kprime;
                const __nv_bfloat16 *bblk = args.Bop + (int64_t)J * np_ * kprime;
                for (int s = 0; s < nk; ++s, ++it) {
                    const uint32_t slot = it % NST, ph = (it / NST) & 1u;
                    if (args.test_drop && it >= 1) {
                        // failure-detection test: the copies of every later stage are
                        // withheld, so the MMA issuer's bounded wait must run out
                        ok = false;
                        break;
                    }
                    if (!mbar_wait(smem_u32(&bars[NST + slot]), ph ^ 1u, args.budget_ns, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t full = smem_u32(&bars[slot]);
                    mbar_expect_tx(full, STAGE_A + stageB_bytes);
                    uint8_t *dst = stages + slot * STAGE_BYTES;
                    bulk_g2s(smem_u32(dst), ablk + (int64_t)s * KST * BM, STAGE_A, full);
                    bulk_g2s(smem_u32(dst + STAGE_A), bblk + (int64_t)s * KST * np_, stageB_bytes, full);
                }
            }
            if (!ok && !args.test_drop) {
                atomicExch(args.status, LDLT_ERR_TIMEOUT_CODE);
                *abort_flag = 1;
            }
            // drain: every issued copy must land before the CTA exits
            for (uint32_t q = (it > NST ? it - NST : 0); q < it; ++q)
                mbar_drain(smem_u32(&bars[q % NST]), (q / NST) & 1u, args.budget_ns);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = make_idesc(BM, np_);
        uint32_t it = 0, tcount = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tcount) {
            const uint32_t buf = tcount & 1u, tph = (tcount >> 1) & 1u;
            if (!mbar_wait(smem_u32(&bars[2 * NST + 2 + buf]), tph ^ 1u, args.budget_ns, abort_flag)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t dtmem = tmem_base + buf * (uint32_t)np_;
            for (int s = 0; s < nk; ++s, ++it) {
                const uint32_t slot = it % NST, ph = (it / NST) & 1u;
                if (!mbar_wait(smem_u32(&bars[slot]), ph, args.budget_ns, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t sa = smem_u32(stages + slot * STAGE_BYTES);
                    const uint32_t sb = sa + STAGE_A;
#pragma unroll
                    for (int kk = 0; kk < KST / 16; ++kk) {
                        // one K=16 step = two core matrices along K
                        const uint64_t ad = make_desc(sa + kk * 2 * (BM * 16), BM * 16, 128);
                        const uint64_t bd = make_desc(sb + kk * 2 * (np_ * 16), np_ * 16, 128);
                        mma_bf16(dtmem, ad, bd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(smem_u32(&bars[NST + slot]));
                }
                __syncwarp();
            }
            if (!ok) break;
            if (lane == 0) mma_commit(smem_u32(&bars[2 * NST + buf]));
            __syncwarp();
        }
        if (!ok) {
            atomicExch(args.status, LDLT_ERR_TIMEOUT_CODE);
            *abort_flag = 1;
            // drain: the MMAs already issued must finish before TMEM is freed
            if (lane == 0) mma_commit(smem_u32(&bars[2 * NST + 4]));
            __syncwarp();
            mbar_drain(smem_u32(&bars[2 * NST + 4]), 0u, args.budget_ns);
        }
    } else {
        // ---------------- epilogue: two groups take alternate tiles ----------------
        // Group g (warps 2+8g .. 9+8g) owns TMEM buffer g.  For its next tile it
        // first gathers the old Schur values S[sigma i][sigma j] into shared
        // memory (this overlaps the MMAs of that tile), then drains the
        // accumulators: recombine the limbs, reduce once mod p, subtract, and
        // store its row's columns with vector stores.  The recombination is
        // bound by instruction latency, so two warps share each TMEM lane
        // quarter (warp w may read lanes 32 (w mod 4) .. +31), each taking
        // half of the tile's columns.
        const int g = (warp - 2) >> 3;       // group
        const int wq = (warp - 2) & 7;       // warp within the group
        const int q = warp & 3;              // TMEM lane quarter this warp may access
        const int hc = wq >> 2;              // column half of the tile this warp drains
        const int row = q * 32 + lane;       // tile row owned in the TMEM phase
        uint32_t *cg = cold + g * BM * CLD;
        const FieldP f = args.f;
        const int L = args.limbs;
        const int mn = m_next;
        const uint64_t bias = args.bias;
        uint32_t tcount = g;
        for (int t = blockIdx.x + g * gridDim.x; t < ntiles; t += 2 * gridDim.x, tcount += 2) {
            int I, J;
            tile_of(tm, t, I, J);
            // -- gather the old values of this tile (rows wq*16 .. wq*16+15) --
            // Asynchronous 4-byte copies, all in flight at once: one memory
            // round trip per tile.  S is only read in this kernel (the new
            // values go to Snext), so the L1-allocating form sees no stale line.
            if (args.upper) {
                // old value of output (i, j) at S[j][i]: warp wq takes the tile's
                // columns wq*8 .. wq*8+7, lanes run along i (contiguous in S)
#pragma unroll 2
                for (int c = 0; c < 8; ++c) {
                    const int jl = wq * 8 + c, j = J * BN + jl;
                    const uint32_t *srow = args.S + (int64_t)j * args.ldS;
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int il = 32 * h + lane, i = I * BM + il;
                        uint32_t *d = cg + il * CLD + jl;
                        if (i < mn && j <= i && j < mn) cp_async4(d, srow + i);
                        else *d = 0u;
                    }
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            } else {
                const int j0 = J * BN + lane, j1 = j0 + 32;
                const int sj0 = j0 < mn ? __ldg(args.sigma + j0) : 0;
                const int sj1 = j1 < mn ? __ldg(args.sigma + j1) : 0;
                const int ilane = I * BM + wq * 16 + (lane & 15);
                const int si_lane = ilane < mn ? __ldg(args.sigma + ilane) : 0;
#pragma unroll 8
                for (int r = 0; r < 16; ++r) {
                    const int i = I * BM + wq * 16 + r;
                    const int si = __shfl_sync(0xffffffffu, si_lane, r);
                    const uint32_t *srow = args.S + (int64_t)si * args.ldS;
                    const int rr = wq * 16 + r;
                    uint32_t *d0 = cg + rr * CLD + lane, *d1 = d0 + 32;
                    if (i < mn && j0 <= i && j0 < mn) cp_async4(d0, srow + sj0);
                    else *d0 = 0u;
                    if (i < mn && j1 <= i && j1 < mn) cp_async4(d1, srow + sj1);
                    else *d1 = 0u;
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            }
            asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(GROUP_THREADS) : "memory");
            const uint32_t tph = (tcount >> 1) & 1u;
            if (!mbar_wait(smem_u32(&bars[2 * NST + g]), tph, args.budget_ns, abort_flag)) {
                atomicExch(args.status, LDLT_ERR_TIMEOUT_CODE);
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)g * (uint32_t)np_;
            const int i = I * BM + row;
            uint32_t *drow = args.Snext + (int64_t)i * args.ldS;
            const uint32_t *crow = cg + row * CLD;
#pragma unroll 1
            for (int c0 = hc * (BN / 2); c0 < (hc + 1) * (BN / 2); c0 += 8) {
                uint32_t r[4][8];
                tmem_ld8(tbase + (uint32_t)(0 * BN + c0), r[0]);
                if (L > 1) tmem_ld8(tbase + (uint32_t)(1 * BN + c0), r[1]);
                if (L > 2) tmem_ld8(tbase + (uint32_t)(2 * BN + c0), r[2]);
                if (L > 3) tmem_ld8(tbase + (uint32_t)(3 * BN + c0), r[3]);
                tmem_wait_ld();
                uint32_t o[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    int64_t v = (int64_t)__float2int_rn(__uint_as_float(r[0][e]));
                    if (L > 1) v += (int64_t)__float2int_rn(__uint_as_float(r[1][e])) << 8;
                    if (L > 2) v += (int64_t)__float2int_rn(__uint_as_float(r[2][e])) << 16;
                    if (L > 3) v += (int64_t)__float2int_rn(__uint_as_float(r[3][e])) << 24;
                    o[e] = fp_sub(crow[c0 + e], fp_reduce64_fold((uint64_t)(v + (int64_t)bias), f), f);
                }
                const int jb = J * BN + c0;
                if (args.upper) {
                    // S[j][i]: the lanes' consecutive rows i make each store one line
                    if (i < mn) {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (jb + e <= i && jb + e < mn) args.Snext[(int64_t)(jb + e) * args.ldS + i] = o[e];
                    }
                } else if (i < mn) {
                    if (jb + 7 <= i && jb + 7 < mn) {
                        uint4 *dst = (uint4 *)(drow + jb);
                        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
                        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (jb + e <= i && jb + e < mn) drow[jb + e] = o[e];
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&bars[2 * NST + 2 + g]));
            asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(GROUP_THREADS) : "memory");
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base));
}

// ---------------------------------------------------------------------------
// operand preparation (split_write and its digit helpers: tc_split.cuh)
// ---------------------------------------------------------------------------
// One thread per (row i, group of 8 columns k..k+7).
__global__ void split_tc_kernel(const SplitArgs a)
{
    if (!step_live(a.ls, a.out)) return;
    const int m_next = a.out->m_next, np = a.out->np;
    if (np == 0) {
        compact_rows(a.S, a.ldS, a.sigma, m_next, a.Snext, blockIdx.y * gridDim.x + blockIdx.x,
                     gridDim.x * gridDim.y);
        return;
    }
    if (m_next == 0) return;
    const int kpad = (np + 63) / 64 * 64, rows = (m_next + BM - 1) / BM * BM, kprime = a.la * kpad;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k0 = blockIdx.y * 8;
    if (i >= rows || k0 >= kpad) return;
    const FieldP f = a.f;
    uint32_t g[10];  // g[1 + e] = G[i][k0 + e], e in [-1, 8]
#pragma unroll
    for (int e = 0; e < 10; ++e) {
        const int k = k0 - 1 + e;
        g[e] = (i < m_next && k >= 0 && k < np) ? a.LpC[(int64_t)k * a.ldL + a.sigma[i]] : 0u;
    }
    int32_t gd_bal[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        uint32_t v = 0;
        if (k < np) {
            const uint32_t ek = a.out->eval[k];
            if (ek != 0) v = fp_mul(ek, g[e + 2], f);
            else if (k > 0 && a.out->eval[k - 1] != 0)
                v = fp_add(fp_mul(a.out->eval[k - 1], g[e], f), fp_mul(a.out->dval[k], g[e + 1], f), f);
            else v = fp_mul(a.out->dval[k], g[e + 1], f);
        }
        gd_bal[e] = balanced(v, f.p);
    }
    uint32_t gk[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) gk[e] = g[e + 1];
    split_write(a, i, k0, kpad, kprime, rows, gd_bal, gk);
}

}  // namespace

// Number of signed 8-bit digits so that every balanced residue |x| <= (p-1)/2
// has a top digit of magnitude at most 128.
int tc_limbs(uint32_t p)
{
    const int64_t h = (int64_t)(p - 1) / 2;
    for (int L = 1; L <= 4; ++L) {
        int64_t lowmax = 0, scale = 1;
        for (int u = 0; u < L - 1; ++u) {
            lowmax += 128 * scale;
            scale *= 256;
        }
        // |top| <= (h + lowmax) / scale
        if ((h + lowmax) / scale <= 128) return L;
    }
    return -1;
}

// Digits of the A side: base 512 when it needs fewer digits than base 256
// (|digit| <= 256 stays exact in bf16; the accumulation bound above allows
// L_A <= 3 with base 512), else the base-256 count.  Returns the count and
// the base's bit width.
int tc_limbs_a(uint32_t p, int *shift)
{
    const int lb = tc_limbs(p);
    const int64_t h = (int64_t)(p - 1) / 2;
    for (int L = 1; L <= 3 && L < lb; ++L) {
        int64_t lowmax = 0, scale = 1;
        for (int u = 0; u < L - 1; ++u) {
            lowmax += 256 * scale;
            scale *= 512;
        }
        if ((h + lowmax) / scale <= 256) {
            *shift = 9;
            return L;
        }
    }
    *shift = 8;
    return lb;
}

int tc_bn(int limbs) { (void)limbs; return BN; }

size_t tc_operand_bytes(int64_t n, int limbs)
{
    const int64_t rows = round_up(n, BM);
    const int64_t kprime = (int64_t)limbs * KP_MAX;
    const int64_t nprime = (int64_t)limbs * tc_bn(limbs);
    const int64_t aBytes = rows * kprime * 2;
    const int64_t bBytes = (rows / tc_bn(limbs)) * nprime * kprime * 2;
    return (size_t)round_up(aBytes, 256) + (size_t)round_up(bBytes, 256);
}

cudaError_t launch_split_tc(const uint32_t *LpC, int64_t ldL, const int *sigma, int64_t n,
                            const LoopState *ls, const PanelOut *out, FieldP f, int limbs, void *Aop,
                            void *Bop, const uint32_t *S, int64_t ldS, uint32_t *Snext, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    SplitArgs a;
    a.LpC = LpC; a.ldL = ldL; a.sigma = sigma;
    int ash = 8;
    a.lb = limbs; a.la = tc_limbs_a(f.p, &ash); a.ash = ash; a.bn = tc_bn(limbs);
    a.nprime = limbs * a.bn;
    a.ls = ls; a.out = out; a.f = f;
    a.S = S; a.ldS = ldS; a.Snext = Snext;
    uint64_t w = 1;
    for (int u = 0; u < 4; ++u) {
        a.wbase[u] = (uint32_t)(w % f.p);
        w = (w << ash) % f.p;
    }
    a.Aop = (__nv_bfloat16 *)Aop;
    a.Bop = (__nv_bfloat16 *)Bop;
    // sized for the largest update (n rows, KP_MAX columns); surplus threads return
    dim3 grid((unsigned)((round_up(n, BM) + 127) / 128), KP_MAX / 8);
    split_tc_kernel<<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

SplitArgs tc_split_args(FieldP f, int limbs, void *Aop, void *Bop)
{
    SplitArgs a;
    a.LpC = nullptr; a.ldL = 0; a.sigma = nullptr;
    int ash = 8;
    a.lb = limbs; a.la = tc_limbs_a(f.p, &ash); a.ash = ash; a.bn = tc_bn(limbs);
    a.nprime = limbs * a.bn;
    a.ls = nullptr; a.out = nullptr; a.f = f;
    a.S = nullptr; a.ldS = 0; a.Snext = nullptr;
    uint64_t w = 1;
    for (int u = 0; u < 4; ++u) {
        a.wbase[u] = (uint32_t)(w % f.p);
        w = (w << ash) % f.p;
    }
    a.Aop = (__nv_bfloat16 *)Aop;
    a.Bop = (__nv_bfloat16 *)Bop;
    return a;
}


cudaError_t launch_syrdk_tc(const uint32_t *S, int64_t ldS, const int *sigma, const LoopState *ls,
                            const PanelOut *out, const void *Aop, const void *Bop, int limbs, FieldP f,
                            uint32_t *Snext, int64_t budget_ns, int32_t *status, int num_sms,
                            int test_drop, cudaStream_t st, int upper)
{
    TcArgs a;
    a.upper = upper;
    a.S = S; a.ldS = ldS; a.sigma = sigma; a.ls = ls; a.out = out;
    a.Aop = (const __nv_bfloat16 *)Aop; a.Bop = (const __nv_bfloat16 *)Bop;
    int ash = 8;
    a.limbs = limbs; a.bn = tc_bn(limbs); a.nprime = limbs * a.bn; a.la = tc_limbs_a(f.p, &ash);
    a.f = f;
    a.bias = ((((uint64_t)1 << 50) / f.p) + 1) * (uint64_t)f.p;
    a.Snext = Snext; a.budget_ns = budget_ns; a.status = status; a.test_drop = test_drop;
    a.nst = NST;
    const size_t smem = 1024 + (size_t)NST * STAGE_BYTES + (size_t)2 * BM * CLD * 4 + 256;
    cudaError_t err = cudaFuncSetAttribute(syrdk_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    // persistent: one CTA per SM, the tile count is read on the device
    syrdk_tc_kernel<<<num_sms, TC_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}
