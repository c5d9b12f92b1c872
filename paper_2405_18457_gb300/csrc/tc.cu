// tcgen05 (sm_103a) fused kernel-matrix product  Y = alpha * K(X1, X2) V + beta * Y + diag.
//
// Flash-attention-like tiling: one CTA owns 128 output rows and streams 128-wide
// column tiles.  Per column tile:
//   GEMM1 (tensor cores, fp16 x fp16 -> fp32 in TMEM):  S = PA_I . PB_J^T, where the
//         prepared operands make S_ij the kernel's exponent argument directly
//         (scaled squared distance, norm terms and the hi/lo split folded in);
//   exp   (4 warps, one TMEM lane = one row each): k'_ij = kappa(S_ij) on MUFU,
//         packed to fp16 and written back over S in TMEM (K never leaves the SM);
//   GEMM2 (tensor cores, A = k' from TMEM, B = V16_J from SMEM): Y_I += K'_IJ V_J.
// A warp-specialised pipeline overlaps them: warp 0 issues TMA loads of PB/V16
// tiles into a ring of shared-memory stages, warp 1 issues tcgen05.mma (one
// thread), warps 4-7 evaluate the kernel and run the epilogue.  Two S buffers in
// TMEM let GEMM1 of tile j+1 run while tile j is being exponentiated.  Every
// mbarrier wait is bounded (about 2 s); on time-out the kernel records an error
// flag, skips the remaining work, releases its tensor memory and returns.
//
// Operand preparation (per call, O(n d)):
//   a_i = x_i / l (ARD scaling), n_i = ||a_i||^2, c the kernel-specific factor
//   (RBF: c = -log2(e)/2 so that k = s_f^2 2^S; Matern-3/2: c = 3 log2(e)^2 so
//   that sqrt(S) = sqrt(3) r log2(e)).  With h(.) = fp16 rounding and
//   l(x) = h(x - h(x)):
//     PA_i = [h(-2c a_i/s), h(-2c a_i/s), l(-2c a_i/s), h(c n_i/s), l(c n_i/s), 1, 1, 0...]
//     PB_j = [h(a_j),       l(a_j),       h(a_j),       1,          1, h(c n_j/s), l(c n_j/s), 0...]
//   so that PA_i . PB_j = (c r_ij^2)/s to ~2^-22 relative of c max(n) (the lo x lo
//   term is dropped), s a power of two that keeps every fp16 entry < 2^14.
//   V is stored as fp16 per column, scaled by a power of two so its largest
//   magnitude lies in [1, 2); the scale is undone in FP32 in the epilogue.
#include "gp_internal.cuh"
#include "tcgen05.cuh"

#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <cmath>
#include <string>
#include <tuple>
#include <vector>

namespace gp {

namespace {

constexpr int TM = 128;          // output rows per CTA
constexpr int TN = 128;          // columns per tile
constexpr int MAX_STAGES = 6;  // gradient kernel: depth of the PB/W ring
constexpr int MAX_B3 = 8;      // gradient kernel: depth of the [A | A^2] ring
constexpr int MAX_RING = 8;    // product kernel: slots per ring (barrier arrays are sized for this)
constexpr int NTHREADS = 416;     // gradient kernel: producer, 3 MMA issuers, 2 x 4 evaluation warps, producer
constexpr int kPersist = -1;       // split code of the persistent product schedule
constexpr int MVM_THREADS = 384;  // product kernel: producer, MMA, 2 idle, 2 x 4 evaluation warps
constexpr int kMaxRhsPerPass = 128;  // right-hand sides per product pass (TMEM columns 384..511)
constexpr int kPersistMaxGrid = 256;  // persistent schedule: at most this many CTAs (d^T y partials per column)
constexpr int kSplitGroup = 8;       // split form: tiles per tensor-memory accumulation group
constexpr int kSplitMaxRpad = 80;    // split form: padded right-hand sides per pass (256 + 3 R_pad <= 512)
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// Set (to 1) by any tensor-core kernel whose bounded wait gave up; read and cleared by the
// host (tc_timeout_status).
__device__ int g_tc_timeout = 0;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// k / s_f^2 from the tile value S (the kernel's exponent argument / s; SCALED
// multiplies by s, skipped when the preparation chose s = 1).
template <int KIND, bool SCALED>
__device__ __forceinline__ float kernel_of(float S, float dscale) {
    const float v = SCALED ? S * dscale : S;
    if (KIND == GP_RBF) {
        return ex2_approx(fminf(v, 0.0f));
    } else {
        float u = fmaxf(v, 1e-30f);
        float q = u * rsqrt_approx(u);  // sqrt(3) r log2(e)
        return fmaf(q, kLn2, 1.0f) * ex2_approx(-q);
    }
}

// 32 tile values of one row -> 16 packed fp16 pairs of k / s_f^2.
template <int KIND, bool SCALED>
__device__ __forceinline__ void eval_chunk(const uint32_t (&r)[32], uint32_t (&pk)[16], float dscale) {
#pragma unroll
    for (int e = 0; e < 16; ++e)
        pk[e] = pack_half2(kernel_of<KIND, SCALED>(__uint_as_float(r[2 * e]), dscale),
                           kernel_of<KIND, SCALED>(__uint_as_float(r[2 * e + 1]), dscale));
}

// 64 tile values of one row -> 32 packed fp16 pairs of k / s_f^2.
template <int KIND, bool SCALED>
__device__ __forceinline__ void eval_chunk64(const uint32_t (&r)[64], uint32_t (&pk)[32], float dscale) {
#pragma unroll
    for (int e = 0; e < 32; ++e)
        pk[e] = pack_half2(kernel_of<KIND, SCALED>(__uint_as_float(r[2 * e]), dscale),
                           kernel_of<KIND, SCALED>(__uint_as_float(r[2 * e + 1]), dscale));
}

// 32 tile values of one row -> k / s_f^2 as 16 packed fp16 pairs of its high part h(k) and 16 of
// its low part h(k - h(k)) (the split form of the product: k = high + low to about 2^-22).
template <int KIND, bool SCALED>
__device__ __forceinline__ void eval_chunk_split(const uint32_t (&r)[32], uint32_t (&ph)[16], uint32_t (&pl)[16],
                                                 float dscale) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const float k0 = kernel_of<KIND, SCALED>(__uint_as_float(r[2 * e]), dscale);
        const float k1 = kernel_of<KIND, SCALED>(__uint_as_float(r[2 * e + 1]), dscale);
        const __half2 h = __floats2half2_rn(k0, k1);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(k0 - hf.x, k1 - hf.y);
        ph[e] = *reinterpret_cast<const uint32_t *>(&h);
        pl[e] = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// Kernel values of one 128-column tile of this thread's row, written over the S columns at taS
// once read.  Plain form: two halves of 64 columns, each to 32 packed columns at taS + 32 half
// (one 64-column load and one 32-column store per half, fewer tensor-memory instructions
// competing with the MMA issue).  Split form: four quarters of 32 columns, quarter q to
// high parts at taS + 32 q and low parts at taS + 32 q + 16.
template <int KIND, bool SPLIT>
__device__ __forceinline__ void eval_tile(uint32_t taS, bool unit, float dsc) {
    if constexpr (!SPLIT) {
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            uint32_t r[64];
            tmem_ld64(taS + half * 64, r);
            tmem_ld_wait();
            uint32_t pk[32];
            if (unit)
                eval_chunk64<KIND, false>(r, pk, dsc);
            else
                eval_chunk64<KIND, true>(r, pk, dsc);
            tmem_st32(taS + half * 32, pk);
        }
    } else {
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            uint32_t r[32];
            tmem_ld32(taS + q * 32, r);
            tmem_ld_wait();
            uint32_t ph[16], pl[16];
            if (unit)
                eval_chunk_split<KIND, false>(r, ph, pl, dsc);
            else
                eval_chunk_split<KIND, true>(r, ph, pl, dsc);
            tmem_st16(taS + q * 32, ph);
            tmem_st16(taS + q * 32 + 16, pl);
        }
    }
}

// GEMM2 of one tile: Y += P V over the tile's 128 columns in K = 16 steps (A = kernel values
// in tensor memory at aP, B = the V tile's 64-column atoms in shared memory at dv).  Split form:
// Y += P_hi V_hi + P_hi V_lo + P_lo V_hi (the low x low term, about 2^-22 relative, dropped),
// V_lo in atoms 2 and 3 of the slot.  acc0: accumulate into Y from the first step on.
template <bool SPLIT>
__device__ __forceinline__ void gemm2_tile(uint32_t tY, uint32_t aP, uint64_t dv, uint32_t va_units, uint32_t id2,
                                           bool acc0) {
#pragma unroll
    for (int k = 0; k < TN / 16; ++k) {
        const uint32_t kv = (uint32_t)(k >> 2), ko = (uint32_t)(k & 3) * 2;
        const uint32_t acc = (acc0 || k > 0) ? 1u : 0u;
        if constexpr (!SPLIT) {
            mma_ts(tY, aP + k * 8, dv + kv * va_units + ko, id2, acc);
        } else {
            const uint32_t aH = aP + (uint32_t)(k >> 1) * 32 + (uint32_t)(k & 1) * 8, aL = aH + 16;
            const uint64_t bH = dv + kv * va_units + ko, bL = dv + (2 + kv) * va_units + ko;
            mma_ts(tY, aH, bH, id2, acc);
            mma_ts(tY, aH, bL, id2, 1u);
            mma_ts(tY, aL, bH, id2, 1u);
        }
    }
}

struct KParams {
    int R, R_pad, KD;
    int npb, nv;         // depths of the PB-tile and V-tile shared-memory rings
    int64_t n1;          // output rows
    int64_t col_tiles;   // 128-wide column tiles over the (padded) column set
    int nsplit;
    float sf2, alpha, beta, diag_coef;
    const float *vinv;   // per right-hand side: 1 / (power-of-two scale of V16)
    const float *dscale; // device scalar s (see operand preparation)
    const float *Vd;
    int64_t ldvd, drow0, ndiag;
    float *Y;
    int64_t ldy;
    float *partial;      // nsplit > 1: partial[split][c][i]; persistent: partial[slot][c][row in tile]
    const int *done;
    int *err;
    // persistent schedule (single problem): CTA b takes the (row tile, column tile) pairs
    // [T b / G, T (b+1) / G) in row-major order, T = ptotal, G = pgrid = gridDim.x; a run of
    // pairs in one row tile is a segment.  Only a CTA's first and last segments can miss part
    // of their row tile; such a segment writes its sums to slot 2 b (first) or 2 b + 1 (last),
    // and the last CTA to finish a piece of the row tile combines the slots (see pcnt).
    int persist;
    int64_t ptotal;
    int pgrid;
    // grouped mode (a batch of independent GPs): one work item per CTA
    const BItem *items;     // null: single problem, grid = row tiles x splits
    const BMember *members;
    const int *mdone;
    // single mode, column panels: PB rows start at *col0_dev (device-resident offset)
    const int64_t *col0_dev;
    int diag_from_col0;     // diagonal rows start at *col0_dev, clipped to ncols_total
    int64_t ncols_total;
    // persistent schedule: arrival counters of the shared row tiles' pieces (8 per row tile;
    // the high 40 bits the launch's generation pgen, the low 24 bits the arrivals), and
    // optionally the partial sums d^T y per column and CTA (dotpart[c * G + b], d = dotv with
    // stride lddv)
    unsigned long long *pcnt;
    unsigned long long pgen;
    const float *dotv;
    int64_t lddv;
    double *dotpart;
};

// CTA of the persistent schedule that takes pair g (CTA b takes [T b / G, T (b + 1) / G)).
__device__ __forceinline__ int64_t cta_of_pair(int64_t g, int64_t T, int G) { return ((g + 1) * G + T - 1) / T - 1; }

// Arrival on a shared row tile's piece counter; 1 for the arrival that completes `need` in this
// launch's generation.  A counter whose generation is another launch's (an earlier launch, an
// aborted one, or whatever a new workspace held: it matches the 40-bit generation by chance with
// probability 2^-40) counts from zero.  Each retry means another CTA's arrival landed first (a
// CTA arrives once per piece and launch), so the loop is short; it is bounded all the same.
constexpr int kCountBits = 24;  // arrivals per piece <= the persistent grid (256)
__device__ __forceinline__ int arrive_last(unsigned long long *cnt, unsigned long long gen, unsigned need,
                                           volatile int *err) {
    constexpr unsigned long long kMask = (1ull << kCountBits) - 1ull;
    unsigned long long old = atomicAdd(cnt, 0ull);
    for (int tries = 0; tries < 4096; ++tries) {
        const unsigned now = ((old >> kCountBits) == gen) ? (unsigned)(old & kMask) : 0u;
        const unsigned long long nw = (gen << kCountBits) | (unsigned long long)(now + 1);
        const unsigned long long seen = atomicCAS(cnt, old, nw);
        if (seen == old) return (now + 1 == need) ? 1 : 0;
        old = seen;
    }
    *err = 1;
    return 0;
}

// KAT: 64-wide atoms of the distance contraction (KD / 64); PERSIST: the persistent schedule
// (single problem; a separate instantiation so that the other schedules keep their code).
template <int KIND, int KAT, bool PERSIST = false, bool SPLIT = false>
__global__ void __launch_bounds__(MVM_THREADS, 1)
    tc_mvm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ CUtensorMap mapV, const KParams p) {
    if (p.done && *p.done) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // persistent schedule: d^T y sums per evaluation warp and owned column (4 KB)
    __shared__ double s_dot[PERSIST ? 8 : 1][PERSIST ? 64 : 1];
    const int katoms = p.KD / 64;
    const int R_pad = p.R_pad;
    const int NPB = p.npb, NV = p.nv;
    const uint32_t a_bytes = (uint32_t)TM * p.KD * 2;
    const uint32_t b_bytes = (uint32_t)TN * p.KD * 2;
    const uint32_t v_atom = (uint32_t)R_pad * 128;
    const uint32_t v_bytes = (SPLIT ? 4 : 2) * v_atom;  // split form: high then low atoms
    // Two independent rings: PB tiles are needed by GEMM1 about two tiles before the
    // V tiles are needed by GEMM2, and each ring slot is released as soon as its own
    // GEMM has read it, so the loads run several tiles ahead of the tensor cores.
    uint8_t *sA = smem;
    uint8_t *sPB = smem + a_bytes;
    uint8_t *sVr = sPB + (size_t)NPB * b_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sVr + (size_t)NV * v_bytes);
    uint64_t *a_full = bars;
    uint64_t *pb_full = bars + 1;
    uint64_t *pb_empty = pb_full + MAX_RING;
    uint64_t *v_full = pb_empty + MAX_RING;
    uint64_t *v_empty = v_full + MAX_RING;
    // Three tile buffers in tensor memory, each holding S (fp32) and then, written over
    // its first 64 columns, the packed fp16 kernel values P of the same tile.
    uint64_t *t_full = v_empty + MAX_RING;  // GEMM1 of a tile landed in buffer b
    uint64_t *t_kval = t_full + 3;          // the evaluation warpgroup wrote P into buffer b
    uint64_t *t_free = t_kval + 3;          // GEMM2 has consumed buffer b
    uint64_t *y_full = t_free + 3;
    uint64_t *y_empty = y_full + 1;  // persistent: the evaluation threads have read Y
    uint64_t *a_empty = y_empty + 1; // persistent: GEMM1 is done with the row operand
    // split form: GEMM2 accumulates groups of kSplitGroup tiles into two alternating buffers,
    // which the evaluation warps add into a running FP32 sum (yg_full: a group's GEMM2 done;
    // yg_empty: its buffer read out)
    uint64_t *yg_full = a_empty + 1;
    uint64_t *yg_empty = yg_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(yg_empty + 2);
    volatile int *s_err = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Work of this CTA: rows [row0, row0 + 128) of PA against ntiles column tiles of PB
    // starting at tile tb0 (V16 tile tv0); output rows are local rows ioff + lane row
    // of the vectors at Yp.
    int64_t row0, tb0, tv0, ioff, pb_off = 0;
    int ntiles;
    int64_t n1 = p.n1, ldy = p.ldy, ldvd = p.ldvd, drow0 = p.drow0, ndiag = p.ndiag;
    float sf2 = p.sf2, diag_coef = p.diag_coef, dsc;
    const float *vinv = p.vinv, *Vd = p.Vd;
    float *Yp = p.Y;
    if constexpr (PERSIST) {
        const int64_t g0 = p.ptotal * blockIdx.x / gridDim.x, g1 = p.ptotal * (blockIdx.x + 1) / gridDim.x;
        row0 = (g0 / p.col_tiles) * TM;  // first segment's rows; later segments follow row by row
        tb0 = g0;                        // global pair index of local tile 0
        tv0 = 0;
        ntiles = (int)(g1 - g0);
        ioff = row0;
        dsc = *p.dscale;
        if (p.col0_dev) {
            pb_off = *p.col0_dev;
            if (p.diag_from_col0) {
                drow0 = pb_off;
                ndiag = min(ndiag, p.ncols_total - pb_off);
            }
        }
    } else if (p.items) {
        const BItem itm = p.items[blockIdx.x];
        if (p.mdone && p.mdone[itm.member]) return;
        const BMember &m = p.members[itm.member];
        row0 = (int64_t)itm.row_tile * TM;
        tb0 = itm.pb_tile;
        tv0 = itm.v_tile;
        ntiles = itm.ntiles;
        ioff = row0 - m.rb;
        n1 = m.n;
        ldy = ldvd = ndiag = m.n;
        drow0 = 0;
        sf2 = m.sf2;
        diag_coef = p.diag_coef * m.sigma2;
        dsc = m.dscale;
        vinv = p.vinv + (int64_t)itm.member * R_pad;
        Yp = p.Y + m.vo;
        Vd = p.Vd ? p.Vd + m.vo : nullptr;
    } else {
        row0 = (int64_t)blockIdx.x * TM;
        const int64_t per = cdiv(p.col_tiles, p.nsplit);
        tb0 = (int64_t)blockIdx.y * per;
        const int64_t t1 = min(p.col_tiles, tb0 + per);
        ntiles = (int)max((int64_t)0, t1 - tb0);
        tv0 = tb0;
        ioff = row0;
        dsc = *p.dscale;
        if (p.col0_dev) {
            pb_off = *p.col0_dev;
            if (p.diag_from_col0) {
                drow0 = pb_off;
                ndiag = min(ndiag, p.ncols_total - pb_off);
            }
        }
    }

    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        for (int s = 0; s < MAX_RING; ++s) {
            mbar_init(&pb_full[s], 1);
            mbar_init(&pb_empty[s], 1);
            mbar_init(&v_full[s], 1);
            mbar_init(&v_empty[s], 1);
        }
        for (int b = 0; b < 3; ++b) {
            mbar_init(&t_full[b], 1);
            mbar_init(&t_kval[b], 128);
            mbar_init(&t_free[b], 1);
        }
        mbar_init(y_full, 1);
        mbar_init(y_empty, 256);
        mbar_init(a_empty, 1);
        for (int k = 0; k < 2; ++k) {
            mbar_init(&yg_full[k], 1);
            mbar_init(&yg_empty[k], 256);
        }
        *s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // Tensor memory: tile buffers 0..2 at columns 0 / 128 / 256 (S fp32; P packed fp16 over
    // its first 64 columns), the Y accumulator at 384 (R_pad <= 128 columns).
    const uint32_t tmem = *tmem_slot;
    const uint32_t tS0 = tmem, tY = tmem + 384;
    // Split form (single segment): two tile buffers at columns 0 / 128, the two group
    // accumulators at 256 and 256 + R_pad, the running sum at 256 + 2 R_pad (R_pad <= 80).
    constexpr int NB = SPLIT ? 2 : 3;  // tile buffers
    const uint32_t tDg = tmem + 256, tYs = tmem + 256 + 2 * (uint32_t)R_pad;
    if constexpr (!PERSIST) {
        if (warp == 0 && ntiles > 0) {
            // ------------------------------------------------ TMA producer: row operand + PB ring
            const bool leader = elect_one();
            if (leader) {
                mbar_expect_tx(a_full, a_bytes);
                for (int ka = 0; ka < katoms; ++ka) tma_load_2d(sA + ka * (TM * 128), &mapA, a_full, ka * 64, (int)row0);
            }
            for (int it = 0; it < ntiles; ++it) {
                const int s = it % NPB;
                if (it >= NPB && !mbar_wait_warp(&pb_empty[s], ((it / NPB) - 1) & 1, s_err)) break;
                const int j0 = (int)((tb0 + it) * TN + pb_off);
                uint8_t *sB = sPB + (size_t)s * b_bytes;
                if (leader) {
                    mbar_expect_tx(&pb_full[s], b_bytes);
                    for (int ka = 0; ka < katoms; ++ka)
                        tma_load_2d(sB + ka * (TN * 128), &mapB, &pb_full[s], ka * 64, j0);
                }
            }
        } else if (warp == 2 && ntiles > 0) {
            // ------------------------------------------------ TMA producer: V ring
            const bool leader = elect_one();
            for (int it = 0; it < ntiles; ++it) {
                const int s = it % NV;
                if (it >= NV && !mbar_wait_warp(&v_empty[s], ((it / NV) - 1) & 1, s_err)) break;
                const int j0 = (int)((tv0 + it) * TN);
                uint8_t *sV = sVr + (size_t)s * v_bytes;
                if (leader) {
                    mbar_expect_tx(&v_full[s], v_bytes);
                    tma_load_2d(sV, &mapV, &v_full[s], j0, 0);
                    tma_load_2d(sV + v_atom, &mapV, &v_full[s], j0 + 64, 0);
                    if constexpr (SPLIT) {
                        tma_load_2d(sV + 2 * v_atom, &mapV, &v_full[s], j0, R_pad);
                        tma_load_2d(sV + 3 * v_atom, &mapV, &v_full[s], j0 + 64, R_pad);
                    }
                }
            }
        } else if (warp == 1 && ntiles > 0) {
            // ------------------------------------------------ GEMM1 issuer
            // GEMM1 and GEMM2 are issued from two warps (1 and 3): each warp's stream of barrier
            // waits, MMAs and commits is then half as long, and the waits of one overlap the MMAs
            // of the other.  Their MMAs touch disjoint tensor memory (S vs P / Y) and every
            // dependency between them runs through the evaluation warpgroups' barriers; a commit
            // tracks the MMAs of its own thread.  Descriptors are built once and advanced by
            // constant offsets (16-byte units).
            const bool leader = elect_one();
            const uint32_t id1 = idesc_f16(TM, TN);
            const uint64_t dA = sdesc(sA), dPB = sdesc(sPB);
            const uint32_t b_units = b_bytes >> 4;
            bool ok = mbar_wait_warp(a_full, 0, s_err);
            // GEMM1 of tile it into buffer it % NB, once GEMM2 of tile it - NB has consumed it.
            for (int it = 0; ok && it < ntiles; ++it) {
                const int s = it % NPB, b = it % NB;
                if (!mbar_wait_warp(&pb_full[s], (it / NPB) & 1, s_err)) break;
                if (it >= NB && !mbar_wait_warp(&t_free[b], ((it / NB) - 1) & 1, s_err)) break;
                tc_fence_after();
                const uint64_t db = dPB + (uint64_t)s * b_units;
                const uint32_t dS = tS0 + b * 128;
                if (leader) {
#pragma unroll
                    for (int k = 0; k < 4 * KAT; ++k) {
                        constexpr uint32_t a_atom = (TM * 128) >> 4, b_atom = (TN * 128) >> 4;
                        const uint32_t ka = (uint32_t)(k >> 2), ko = (uint32_t)(k & 3) * 2;
                        mma_ss(dS, dA + ka * a_atom + ko, db + ka * b_atom + ko, id1, k > 0 ? 1u : 0u);
                    }
                    mma_commit(&pb_empty[s]);
                    mma_commit(&t_full[b]);
                }
                __syncwarp();
            }
        } else if (warp == 3 && ntiles > 0) {
            // ------------------------------------------------ GEMM2 issuer: Y += P V
            const bool leader = elect_one();
            const uint32_t id2 = idesc_f16(TM, R_pad);
            const uint64_t dV = sdesc(sVr);
            const uint32_t v_units = v_bytes >> 4, va_units = v_atom >> 4;
            for (int it = 0; it < ntiles; ++it) {
                const int s = it % NV, b = it % NB;
                // split form: group gi of kSplitGroup tiles into accumulator gi % 2, restarted once
                // the evaluation warps have read out group gi - 2
                const int gi = it / kSplitGroup;
                const bool gfirst = (it % kSplitGroup) == 0;
                const bool glast = (it % kSplitGroup) == kSplitGroup - 1 || it == ntiles - 1;
                if (SPLIT && gfirst && gi >= 2 && !mbar_wait_warp(&yg_empty[gi & 1], ((gi >> 1) - 1) & 1, s_err))
                    break;
                if (!mbar_wait_warp(&v_full[s], (it / NV) & 1, s_err)) break;
                if (!mbar_wait_warp(&t_kval[b], (it / NB) & 1, s_err)) break;
                tc_fence_after();
                const uint64_t dv = dV + (uint64_t)s * v_units;
                const uint32_t aP = tS0 + b * 128;
                if (leader) {
                    if constexpr (SPLIT)
                        gemm2_tile<SPLIT>(tDg + (uint32_t)(gi & 1) * R_pad, aP, dv, va_units, id2, !gfirst);
                    else
                        gemm2_tile<SPLIT>(tY, aP, dv, va_units, id2, it > 0);
                    mma_commit(&v_empty[s]);
                    mma_commit(&t_free[b]);
                    if (SPLIT && glast) mma_commit(&yg_full[gi & 1]);
                }
                __syncwarp();
            }
            if (leader) mma_commit(y_full);
        } else if (warp >= 4) {
            // ------------------------------------------------ kernel evaluation + epilogue
            // Two warpgroups ping-pong: warpgroup wg evaluates the tiles with it % 2 == wg (in
            // buffer it % 3), so one group evaluates while the other waits on tensor memory.
            // Each thread owns one row: it reads 64 S columns, then writes their 64 kernel
            // values (32 packed columns) over the columns it has just read, so P needs no
            // buffer of its own and the warpgroup never waits for GEMM2.
            const int wg = (warp - 4) >> 2;
            const int wq = warp & 3;  // TMEM lane quarter this warp may access
            const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
            const bool unit = (dsc == 1.0f);
            bool ok = true;
            // split form: read-out of group g's accumulator into the running sum (FP32, rounded
            // to nearest), this warpgroup's alternate 16-column chunks, then release the buffer
            const int ngroups = SPLIT ? (int)cdiv(ntiles, kSplitGroup) : 0;
            int rg = 0;  // next group to read out
            auto readout = [&](int g) {
                if (!ok) return;
                ok = mbar_wait(&yg_full[g & 1], (g >> 1) & 1, s_err);
                if (!ok) return;
                tc_fence_after();
                const uint32_t tD = tDg + (uint32_t)(g & 1) * R_pad + lane_off;
                for (int c0 = 16 * wg; c0 < R_pad; c0 += 32) {
                    uint32_t r[16], q[16];
                    tmem_ld16(tD + c0, r);
                    if (g > 0) tmem_ld16(tYs + lane_off + c0, q);
                    tmem_ld_wait();
                    if (g > 0) {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            r[e] = __float_as_uint(__uint_as_float(r[e]) + __uint_as_float(q[e]));
                    }
                    tmem_st16(tYs + lane_off + c0, r);
                }
                tmem_st_wait();
                tc_fence_before();
                mbar_arrive(&yg_empty[g & 1]);
            };
            for (int it = wg; it < ntiles; it += 2) {
                const int b = it % NB;
                if (!mbar_wait(&t_full[b], (it / NB) & 1, s_err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                eval_tile<KIND, SPLIT>(tS0 + b * 128 + lane_off, unit, dsc);
                if (!ok) break;
                tmem_st_wait();
                tc_fence_before();
                mbar_arrive(&t_kval[b]);
                if constexpr (SPLIT) {
                    // groups in which this warpgroup has no tile left
                    while (rg < ngroups && it + 2 >= min(ntiles, (rg + 1) * kSplitGroup)) readout(rg++);
                }
            }
            if constexpr (SPLIT) {
                while (ok && rg < ngroups) readout(rg++);
            }
            // epilogue: Y rows from TMEM lanes, one row per thread; the two warpgroups
            // take alternate 16-column chunks of the right-hand sides (the split form's running
            // sum holds this warpgroup's own chunks)
            if (!SPLIT && ok && ntiles > 0) ok = mbar_wait(y_full, 0, s_err);
            if (ok && ntiles > 0) {
                tc_fence_after();
                const int64_t i = ioff + wq * 32 + lane;
                const bool diag = diag_coef != 0.0f && i >= drow0 && i < drow0 + ndiag;
                for (int c0 = 16 * wg; c0 < R_pad; c0 += 32) {
                    uint32_t r[16];
                    tmem_ld16((SPLIT ? tYs : tY) + lane_off + c0, r);
                    tmem_ld_wait();
                    if (i < n1) {
                        // the loads of the chunk (scales, diagonal vector) before the first store,
                        // so that they are in flight together (a previous Y, beta != 0, is read
                        // with the store)
                        float v[16], vd[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int c = c0 + e;
                            const bool okc = c < p.R;
                            v[e] = okc ? sf2 * vinv[c] * __uint_as_float(r[e]) : 0.0f;
                            vd[e] = (okc && p.nsplit <= 1 && diag) ? Vd[(int64_t)c * ldvd + (i - drow0)] : 0.0f;
                        }
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int c = c0 + e;
                            if (c >= p.R) break;
                            if (p.nsplit > 1) {
                                p.partial[((int64_t)blockIdx.y * p.R + c) * n1 + i] = v[e];
                            } else {
                                float y = p.alpha * v[e];
                                if (p.beta != 0.0f) y += p.beta * Yp[(int64_t)c * ldy + i];
                                if (diag) y += diag_coef * vd[e];
                                Yp[(int64_t)c * ldy + i] = y;
                            }
                        }
                    }
                }
            }
        }
    } else {
        // Walk over the CTA's tiles: the PB / V tile of local tile it, its segment (row tile
        // relative to the first) and whether it opens or closes the segment, advanced one tile
        // at a time.  Without the persistent schedule a CTA has one segment.
        const int64_t ctiles = p.col_tiles, r_first = row0 / TM;
        struct Walk {
            int64_t ct;  // column tile (persistent) or local offset
            int seg;
        };
        auto walk0 = [&]() { return Walk{PERSIST ? tb0 - r_first * ctiles : 0, 0}; };
        auto walk_next = [&](Walk &w) {
            if (++w.ct == ctiles && PERSIST) {
                w.ct = 0;
                ++w.seg;
            }
        };
        auto tile_pb = [&](const Walk &w, int it) { return PERSIST ? w.ct : tb0 + it; };
        auto tile_v = [&](const Walk &w, int it) { return PERSIST ? w.ct : tv0 + it; };
        auto tile_first = [&](const Walk &w, int it) { return it == 0 || (PERSIST && w.ct == 0); };
        auto tile_last = [&](const Walk &w, int it) { return it == ntiles - 1 || (PERSIST && w.ct == ctiles - 1); };

        if (warp == 0 && ntiles > 0) {
            // ------------------------------------------------ TMA producer: row operand + PB ring
            const bool leader = elect_one();
            Walk w = walk0();
            for (int it = 0; it < ntiles; ++it, walk_next(w)) {
                const int seg = w.seg;
                const int64_t pbt = tile_pb(w, it);
                if (tile_first(w, it)) {
                    // row operand of this segment, once GEMM1 has finished with the previous one
                    if (seg > 0 && !mbar_wait_warp(a_empty, (seg - 1) & 1, s_err)) break;
                    if (leader) {
                        mbar_expect_tx(a_full, a_bytes);
                        const int ra = (int)((r_first + seg) * TM);
                        for (int ka = 0; ka < katoms; ++ka) tma_load_2d(sA + ka * (TM * 128), &mapA, a_full, ka * 64, ra);
                    }
                }
                const int s = it % NPB;
                if (it >= NPB && !mbar_wait_warp(&pb_empty[s], ((it / NPB) - 1) & 1, s_err)) break;
                const int j0 = (int)(pbt * TN + pb_off);
                uint8_t *sB = sPB + (size_t)s * b_bytes;
                if (leader) {
                    mbar_expect_tx(&pb_full[s], b_bytes);
                    for (int ka = 0; ka < katoms; ++ka)
                        tma_load_2d(sB + ka * (TN * 128), &mapB, &pb_full[s], ka * 64, j0);
                }
            }
        } else if (warp == 2 && ntiles > 0) {
            // ------------------------------------------------ TMA producer: V ring
            const bool leader = elect_one();
            Walk w = walk0();
            for (int it = 0; it < ntiles; ++it, walk_next(w)) {
                const int s = it % NV;
                if (it >= NV && !mbar_wait_warp(&v_empty[s], ((it / NV) - 1) & 1, s_err)) break;
                const int j0 = (int)(tile_v(w, it) * TN);
                uint8_t *sV = sVr + (size_t)s * v_bytes;
                if (leader) {
                    mbar_expect_tx(&v_full[s], v_bytes);
                    tma_load_2d(sV, &mapV, &v_full[s], j0, 0);
                    tma_load_2d(sV + v_atom, &mapV, &v_full[s], j0 + 64, 0);
                    if constexpr (SPLIT) {
                        tma_load_2d(sV + 2 * v_atom, &mapV, &v_full[s], j0, R_pad);
                        tma_load_2d(sV + 3 * v_atom, &mapV, &v_full[s], j0 + 64, R_pad);
                    }
                }
            }
        } else if (warp == 1 && ntiles > 0) {
            // ------------------------------------------------ GEMM1 issuer
            // GEMM1 and GEMM2 are issued from two warps (1 and 3): each warp's stream of barrier
            // waits, MMAs and commits is then half as long, and the waits of one overlap the MMAs
            // of the other.  Their MMAs touch disjoint tensor memory (S vs P / Y) and every
            // dependency between them runs through the evaluation warpgroups' barriers; a commit
            // tracks the MMAs of its own thread.  Descriptors are built once and advanced by
            // constant offsets (16-byte units).
            const bool leader = elect_one();
            const uint32_t id1 = idesc_f16(TM, TN);
            const uint64_t dA = sdesc(sA), dPB = sdesc(sPB);
            const uint32_t b_units = b_bytes >> 4;
            // GEMM1 of tile it into buffer it % 3, once GEMM2 of tile it - 3 has consumed it.
            Walk w = walk0();
            for (int it = 0; it < ntiles; ++it, walk_next(w)) {
                const bool last = tile_last(w, it);
                if (tile_first(w, it) && !mbar_wait_warp(a_full, w.seg & 1, s_err)) break;
                const int s = it % NPB, b = it % 3;
                if (!mbar_wait_warp(&pb_full[s], (it / NPB) & 1, s_err)) break;
                if (it >= 3 && !mbar_wait_warp(&t_free[b], ((it / 3) - 1) & 1, s_err)) break;
                tc_fence_after();
                const uint64_t db = dPB + (uint64_t)s * b_units;
                const uint32_t dS = tS0 + b * 128;
                if (leader) {
#pragma unroll
                    for (int k = 0; k < 4 * KAT; ++k) {
                        constexpr uint32_t a_atom = (TM * 128) >> 4, b_atom = (TN * 128) >> 4;
                        const uint32_t ka = (uint32_t)(k >> 2), ko = (uint32_t)(k & 3) * 2;
                        mma_ss(dS, dA + ka * a_atom + ko, db + ka * b_atom + ko, id1, k > 0 ? 1u : 0u);
                    }
                    mma_commit(&pb_empty[s]);
                    mma_commit(&t_full[b]);
                    if (last) mma_commit(a_empty);
                }
                __syncwarp();
            }
        } else if (warp == 3 && ntiles > 0) {
            // ------------------------------------------------ GEMM2 issuer: Y += P V
            const bool leader = elect_one();
            const uint32_t id2 = idesc_f16(TM, R_pad);
            const uint64_t dV = sdesc(sVr);
            const uint32_t v_units = v_bytes >> 4, va_units = v_atom >> 4;
            Walk w = walk0();
            for (int it = 0; it < ntiles; ++it, walk_next(w)) {
                const int seg = w.seg;
                const bool first = tile_first(w, it), last = tile_last(w, it);
                const int s = it % NV, b = it % 3;
                // a new segment restarts the accumulator once the previous one has been read out
                if (first && seg > 0 && !mbar_wait_warp(y_empty, (seg - 1) & 1, s_err)) break;
                if (!mbar_wait_warp(&v_full[s], (it / NV) & 1, s_err)) break;
                if (!mbar_wait_warp(&t_kval[b], (it / 3) & 1, s_err)) break;
                tc_fence_after();
                const uint64_t dv = dV + (uint64_t)s * v_units;
                const uint32_t aP = tS0 + b * 128;
                if (leader) {
                    gemm2_tile<SPLIT>(tY, aP, dv, va_units, id2, !first);
                    mma_commit(&v_empty[s]);
                    mma_commit(&t_free[b]);
                    if (last) mma_commit(y_full);
                }
                __syncwarp();
            }
        } else if (warp >= 4) {
            // ------------------------------------------------ kernel evaluation + epilogue
            // Two warpgroups ping-pong: warpgroup wg evaluates the tiles with it % 2 == wg (in
            // buffer it % 3), so one group evaluates while the other waits on tensor memory.
            // Each thread owns one row: it reads 64 S columns, then writes their 64 kernel
            // values (32 packed columns) over the columns it has just read, so P needs no
            // buffer of its own and the warpgroup never waits for GEMM2.
            const int wg = (warp - 4) >> 2;
            const int wq = warp & 3;  // TMEM lane quarter this warp may access
            const int piece = warp - 4;  // this warp's rows x columns piece of a row tile (of 8)
            const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
            const bool unit = (dsc == 1.0f);
            const bool dot = p.dotpart != nullptr;
            bool ok = true;
            s_dot[piece][lane] = 0.0;
            s_dot[piece][lane + 32] = 0.0;
            __syncwarp();
            // d^T y of the rows this CTA finalises: products of one 16-column chunk, summed over
            // the warp's 32 rows in FP32 and added in FP64 to the warp's slots (chunk k of the
            // warpgroup's columns c0 = 16 wg + 32 k at 16 k)
            auto dot_add = [&](const float (&pr)[16], int k) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    float v = pr[e];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) s_dot[piece][16 * k + e] += (double)v;
                }
            };
            // Final row i of Y for the 16 columns c0 .. c0 + 15 from their product sums v (alpha,
            // beta and diagonal terms), and the products dotv y into pr.  The loads of the chunk
            // are issued before the first store, so that they are in flight together (a previous
            // Y, beta != 0, is read with the store).
            auto finish16 = [&](int64_t i, int c0, const float (&v)[16], float (&pr)[16]) {
                const bool diag = diag_coef != 0.0f && i >= drow0 && i < drow0 + ndiag;
                float vd[16], dv[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int c = c0 + e;
                    const bool okc = i < n1 && c < p.R;
                    vd[e] = (okc && diag) ? Vd[(int64_t)c * ldvd + (i - drow0)] : 0.0f;
                    dv[e] = (okc && dot) ? __ldg(&p.dotv[(int64_t)c * p.lddv + i]) : 0.0f;
                }
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int c = c0 + e;
                    pr[e] = 0.0f;
                    if (i < n1 && c < p.R) {
                        float y = p.alpha * v[e];
                        if (p.beta != 0.0f) y += p.beta * Yp[(int64_t)c * ldy + i];
                        if (diag) y += diag_coef * vd[e];
                        Yp[(int64_t)c * ldy + i] = y;
                        pr[e] = dv[e] * y;
                    }
                }
            };
            // A row tile that several CTAs share: each CTA's warp `piece` has written its rows x
            // columns of the tile's partial sums to its slot; the warp that arrives last on the
            // piece's counter (of any of those CTAs) sums the slots in CTA order and finishes
            // the piece's rows.  The counters carry the launch's 40-bit generation above the count,
            // so a count left by an earlier (aborted) launch restarts at zero.
            auto shared_tile = [&](int64_t r) {
                const int64_t T = p.ptotal;
                const int G = (int)gridDim.x;
                const int64_t bf = cta_of_pair(r * ctiles, T, G), bl = cta_of_pair((r + 1) * ctiles - 1, T, G);
                __threadfence();  // this lane's slot writes, visible before the arrival
                __syncwarp();
                int last = 0;
                if (lane == 0) last = arrive_last(&p.pcnt[r * 8 + piece], p.pgen, (unsigned)(bl - bf + 1), s_err);
                last = __shfl_sync(0xffffffffu, last, 0);
                if (!last) return;
                __syncwarp();  // lane 0's arrival, then every lane's acquire fence and reads
                __threadfence();
                const int s0 = (T * bf / G < r * ctiles) ? 1 : 0;  // the first CTA's slot (its last segment)
                const int row = wq * 32 + lane;
                const int64_t i = r * TM + row;
                for (int c0 = 16 * wg, k = 0; c0 < R_pad; c0 += 32, ++k) {
                    // the slots in CTA order, 16 independent loads per slot
                    float v[16], pr[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] = 0.0f;
                    for (int64_t q = bf; q <= bl; ++q) {
                        const float *src = p.partial + ((q * 2 + (q == bf ? s0 : 0)) * p.R) * TM + row;
                        float t[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            t[e] = (i < n1 && c0 + e < p.R) ? __ldcg(src + (int64_t)(c0 + e) * TM) : 0.0f;
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[e] += t[e];
                    }
                    finish16(i, c0, v, pr);
                    if (dot) dot_add(pr, k);
                }
            };
            // Read-out of segment sg's accumulator: final rows when the segment is a whole row
            // tile, else this CTA's slot of a shared row tile (slot 2 b for its first segment,
            // 2 b + 1 for its last).  Both warpgroups take alternate 16-column chunks, release
            // Y to GEMM2, then (shared tile) arrive on the piece's counter.
            auto epilogue = [&](int sg) {
                if (!ok) return;
                ok = mbar_wait_warp(y_full, sg & 1, s_err);
                if (!ok) return;
                tc_fence_after();
                const int64_t r = r_first + sg;
                const int64_t s0 = max(tb0, r * ctiles), s1 = min(tb0 + ntiles, (r + 1) * ctiles);
                const bool whole = (s0 == r * ctiles) && (s1 == (r + 1) * ctiles);
                const int64_t i = r * TM + wq * 32 + lane;
                for (int c0 = 16 * wg, k = 0; c0 < R_pad; c0 += 32, ++k) {
                    uint32_t rr[16];
                    tmem_ld16(tY + lane_off + c0, rr);
                    tmem_ld_wait();
                    float v[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] = (c0 + e < p.R) ? sf2 * vinv[c0 + e] * __uint_as_float(rr[e]) : 0.0f;
                    if (!whole) {
                        if (i < n1) {
#pragma unroll
                            for (int e = 0; e < 16; ++e)
                                if (c0 + e < p.R)
                                    p.partial[(((int64_t)blockIdx.x * 2 + (sg > 0)) * p.R + c0 + e) * TM + (wq * 32 + lane)] =
                                        v[e];
                        }
                    } else {
                        float pr[16];
                        finish16(i, c0, v, pr);
                        if (dot) dot_add(pr, k);
                    }
                }
                tc_fence_before();
                mbar_arrive(y_empty);
                if (!whole) shared_tile(r);
            };
            const int nseg = ntiles <= 0 ? 0 : (int)((tb0 + ntiles - 1) / ctiles - r_first) + 1;
            int it = wg;
            for (int sg = 0; sg < nseg; ++sg) {
                // this warpgroup's tiles of segment sg, then the segment's read-out
                const int seg_end = (int)min((int64_t)ntiles, (r_first + sg + 1) * ctiles - tb0);
                for (; ok && it < seg_end; it += 2) {
                    const int b = it % 3;
                    if (!mbar_wait_warp(&t_full[b], (it / 3) & 1, s_err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    eval_tile<KIND, SPLIT>(tS0 + b * 128 + lane_off, unit, dsc);
                    if (!ok) break;
                    tmem_st_wait();
                    tc_fence_before();
                    mbar_arrive(&t_kval[b]);
                }
                epilogue(sg);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
    if constexpr (PERSIST) {
        // this CTA's d^T y partial per column: the four warps of the column's warpgroup, in order
        if (p.dotpart && threadIdx.x < p.R) {
            const int c = threadIdx.x, wgc = (c >> 4) & 1, slot = (c >> 5) * 16 + (c & 15);
            double t = 0.0;
            for (int q = 0; q < 4; ++q) t += s_dot[wgc * 4 + q][slot];
            p.dotpart[(int64_t)c * gridDim.x + blockIdx.x] = t;
        }
    }
    if (threadIdx.x == 0 && *s_err && p.err) atomicExch(p.err, 1);
}

// Empty column set or split partial reduction + epilogue.
__global__ void tc_reduce_kernel(KParams p) {
    if (p.done && *p.done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= p.n1) return;
    int64_t drow0 = p.drow0, ndiag = p.ndiag;
    if (p.col0_dev && p.diag_from_col0) {
        drow0 = *p.col0_dev;
        ndiag = min(ndiag, p.ncols_total - drow0);
    }
    float s = 0.0f;
    for (int sp = 0; sp < p.nsplit; ++sp) s += p.partial[((int64_t)sp * p.R + c) * p.n1 + i];
    float y = p.alpha * s;
    if (p.beta != 0.0f) y += p.beta * p.Y[(int64_t)c * p.ldy + i];
    if (p.diag_coef != 0.0f && i >= drow0 && i < drow0 + ndiag)
        y += p.diag_coef * p.Vd[(int64_t)c * p.ldvd + (i - drow0)];
    p.Y[(int64_t)c * p.ldy + i] = y;
}

// ------------------------------------------------------------------ operand preparation
__device__ __forceinline__ void split16(float x, __half *hi, __half *lo) {
    __half h = __float2half_rn(x);
    *hi = h;
    *lo = __float2half_rn(x - __half2float(h));
}

// max over points of c*||a||^2 and of |2 c a_k|  (as float bits, atomicMax on ints)
__global__ void tc_bound_kernel(const KP<float> kp, float c, const float *X, int64_t n, unsigned int *bound,
                                const float *inv_dev) {
    float m = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float nrm = 0.0f, amax = 0.0f;
        for (int k = 0; k < kp.d; ++k) {
            float a = X[i * kp.d + k] * (inv_dev ? inv_dev[k] : kp.inv_ell[k]);
            nrm += a * a;
            amax = fmaxf(amax, fabsf(a));
        }
        m = fmaxf(m, fmaxf(fabsf(c) * nrm, 2.0f * fabsf(c) * amax));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(bound, __float_as_uint(m));
}

// One prepared row (see the header comment): x is the point (d coordinates), a = x / l.
// pa / pb may be null (row or column operand only).
__device__ __forceinline__ void operand_row(const float *x, const float *inv_ell, int d, float c, float inv_s, int KD,
                                            __half *pa, __half *pb) {
    const __half z = __float2half_rn(0.0f), one = __float2half_rn(1.0f);
    float nrm = 0.0f;
    for (int k = 0; k < d; ++k) {
        float a = x[k] * inv_ell[k];
        __half h, l;
        split16(a, &h, &l);
        float ar = __half2float(h) + __half2float(l);  // the value the tensor cores see
        nrm += ar * ar;
        if (pb) {
            pb[k] = h;
            pb[d + k] = l;
            pb[2 * d + k] = h;
        }
        if (pa) {
            __half h2, l2;
            split16(-2.0f * c * inv_s * ar, &h2, &l2);
            pa[k] = h2;
            pa[d + k] = h2;
            pa[2 * d + k] = l2;
        }
    }
    __half nh, nl;
    split16(c * inv_s * nrm, &nh, &nl);
    const int o = 3 * d;
    if (pa) {
        pa[o] = nh;
        pa[o + 1] = nl;
        pa[o + 2] = one;
        pa[o + 3] = one;
        for (int k = o + 4; k < KD; ++k) pa[k] = z;
    }
    if (pb) {
        pb[o] = one;
        pb[o + 1] = one;
        pb[o + 2] = nh;
        pb[o + 3] = nl;
        for (int k = o + 4; k < KD; ++k) pb[k] = z;
    }
}

__device__ __forceinline__ void zero_row(int KD, __half *pa, __half *pb) {
    const __half z = __float2half_rn(0.0f);
    for (int k = 0; k < KD; ++k) {
        if (pa) pa[k] = z;
        if (pb) pb[k] = z;
    }
}

// s = smallest power of two with bound / s <= 2^14
__device__ __forceinline__ float operand_scale(float bnd) {
    float s = 1.0f;
    while (bnd / s > 16384.0f) s *= 2.0f;
    return s;
}

// Writes PA (if PA) and PB (if PB) rows for the point set X (n points, n_pad rows): one warp
// per row, the same values as operand_row.  Lane l splits the coordinates l and l + 32 (d <= 64);
// the row's KD halves are then written as half2 pairs by consecutive lanes (coalesced), each
// lane fetching the split parts of the coordinate a position needs by a shuffle.
__device__ __forceinline__ uint32_t pack2(__half a, __half b) {
    __half2 h = __halves2half2(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ __half lo_half(uint32_t u) { return __ushort_as_half((unsigned short)(u & 0xFFFFu)); }
__device__ __forceinline__ __half hi_half(uint32_t u) { return __ushort_as_half((unsigned short)(u >> 16)); }

// tc_operands_kernel takes one warp per point: 8 points per 256-thread block, at most 32 blocks
// per SM (a grid-strided walk beyond that).
inline unsigned operand_blocks(int64_t n_pad) { return (unsigned)std::min<int64_t>(cdiv(n_pad, 8), 152 * 32); }

__global__ void tc_operands_kernel(const KP<float> kp, float c, const float *X, int64_t n, int64_t n_pad, int KD,
                                   const unsigned int *bound, __half *PA, __half *PB, float *dscale_out,
                                   const float *inv_dev) {
    const float s = operand_scale(__uint_as_float(*bound));
    if (blockIdx.x == 0 && threadIdx.x == 0 && dscale_out) *dscale_out = s;
    const float inv_s = 1.0f / s;
    const int d = kp.d, lane = threadIdx.x & 31;
    const __half z = __float2half_rn(0.0f), one = __float2half_rn(1.0f);
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n_pad; i += nw) {
        // split parts of coordinates lane (A) and lane + 32 (B): (h, l) for PB, (h2, l2) for PA
        uint32_t bA = 0, aA = 0, bB = 0, aB = 0;
        float sq = 0.0f;
        if (i < n) {
            for (int h = 0; h < 2; ++h) {
                const int k = lane + 32 * h;
                if (k >= d) break;
                const float a = X[i * d + k] * (inv_dev ? inv_dev[k] : kp.inv_ell[k]);
                __half hh, ll, h2, l2;
                split16(a, &hh, &ll);
                const float ar = __half2float(hh) + __half2float(ll);  // the value the tensor cores see
                sq = fmaf(ar, ar, sq);
                split16(-2.0f * c * inv_s * ar, &h2, &l2);
                if (h == 0) {
                    bA = pack2(hh, ll);
                    aA = pack2(h2, l2);
                } else {
                    bB = pack2(hh, ll);
                    aB = pack2(h2, l2);
                }
            }
        }
        float nrm = sq;
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        __half nh, nl;
        split16(c * inv_s * nrm, &nh, &nl);
        const int o3 = 3 * d;
        for (int p0 = 2 * lane; p0 < KD; p0 += 64) {
            __half va[2], vb[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int pos = p0 + e;
                // coordinate and segment of this position: [h(a) | l(a) | h(a)] in PB,
                // [h(-2ca/s) | h(-2ca/s) | l(-2ca/s)] in PA
                const int seg = pos < o3 ? pos / d : 3, k = pos < o3 ? pos - seg * d : 0;
                // every lane passes the same variable to a shuffle; lane src holds coordinate k
                const int src = k & 31;
                uint32_t b32 = __shfl_sync(0xffffffffu, bA, src);
                uint32_t a32 = __shfl_sync(0xffffffffu, aA, src);
                if (d > 32) {  // uniform: coordinates 32 .. d-1 live in the second pair
                    const uint32_t b2 = __shfl_sync(0xffffffffu, bB, src);
                    const uint32_t a2 = __shfl_sync(0xffffffffu, aB, src);
                    if (k >= 32) {
                        b32 = b2;
                        a32 = a2;
                    }
                }
                __half pa, pb;
                if (i >= n) {
                    pa = pb = z;
                } else if (pos < o3) {
                    pb = (seg == 1) ? hi_half(b32) : lo_half(b32);
                    pa = (seg == 2) ? hi_half(a32) : lo_half(a32);
                } else if (pos == o3) {
                    pa = nh;
                    pb = one;
                } else if (pos == o3 + 1) {
                    pa = nl;
                    pb = one;
                } else if (pos == o3 + 2) {
                    pa = one;
                    pb = nh;
                } else if (pos == o3 + 3) {
                    pa = one;
                    pb = nl;
                } else {
                    pa = pb = z;
                }
                va[e] = pa;
                vb[e] = pb;
            }
            if (PA) *reinterpret_cast<__half2 *>(PA + i * KD + p0) = __halves2half2(va[0], va[1]);
            if (PB) *reinterpret_cast<__half2 *>(PB + i * KD + p0) = __halves2half2(vb[0], vb[1]);
        }
    }
}

// ------------------------------------------------------------------ batches (grouped operands)
// Per member bound (float bits, atomicMax) over its chunks: max of c ||a||^2 and 2 c |a_k|.
__global__ void tc_group_bound_kernel(BMember *mem, const BChunk *chunks, int nchunks, const float *X, float c) {
    __shared__ float red[8];
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const BChunk k = chunks[ch];
        const BMember &m = mem[k.member];
        const int d = m.d;
        float mx = 0.0f;
        for (int r = threadIdx.x; r < kBatchChunk; r += blockDim.x) {
            const int64_t i = (int64_t)k.start + r;
            if (i >= m.n) break;
            const float *x = X + m.xo + i * d;
            float nrm = 0.0f, amax = 0.0f;
            for (int q = 0; q < d; ++q) {
                float a = x[q] * m.inv_ell[q];
                nrm += a * a;
                amax = fmaxf(amax, fabsf(a));
            }
            mx = fmaxf(mx, fmaxf(fabsf(c) * nrm, 2.0f * fabsf(c) * amax));
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
            atomicMax(&mem[k.member].bound, __float_as_uint(t));
        }
        __syncthreads();
    }
}

struct GroupOut {
    __half *PA[3], *PB[3];
    int KD[3];
};

__global__ void tc_group_operands_kernel(BMember *mem, const BChunk *chunks, int nchunks, const float *X, float c,
                                         GroupOut o) {
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const BChunk k = chunks[ch];
        const BMember &m = mem[k.member];
        const float s = operand_scale(__uint_as_float(m.bound));
        if (k.start == 0 && threadIdx.x == 0) mem[k.member].dscale = s;
        const float inv_s = 1.0f / s;
        const int KD = o.KD[m.cls];
        const int64_t n_pad = rup(m.n, TM);
        for (int r = threadIdx.x; r < kBatchChunk; r += blockDim.x) {
            const int64_t i = (int64_t)k.start + r;
            if (i >= n_pad) break;
            __half *pa = o.PA[m.cls] + (m.rb + i) * KD;
            __half *pb = o.PB[m.cls] + (m.rb + i) * KD;
            if (i >= m.n)
                zero_row(KD, pa, pb);
            else
                operand_row(X + m.xo + i * m.d, m.inv_ell, m.d, c, inv_s, KD, pa, pb);
        }
    }
}

// colmax[g][c] = max |V_g[c][i]| over the member's rows (float bits, atomicMax)
__global__ void tc_group_colmax_kernel(const BMember *mem, const BChunk *chunks, int nchunks, const float *V, int R,
                                       int R_pad, unsigned *colmax, const int *mdone) {
    __shared__ float red[8];
    const int c = blockIdx.y;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const BChunk k = chunks[ch];
        if (mdone && mdone[k.member]) continue;
        const BMember &m = mem[k.member];
        const float *v = V + m.vo + (int64_t)c * m.n;
        float mx = 0.0f;
        for (int r = threadIdx.x; r < kBatchChunk; r += blockDim.x) {
            const int64_t i = (int64_t)k.start + r;
            if (i >= m.n) break;
            mx = fmaxf(mx, fabsf(v[i]));
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
            if (t > 0.0f) atomicMax(&colmax[(int64_t)k.member * R_pad + c], __float_as_uint(t));
        }
        __syncthreads();
    }
}

// V16[c][cb + i] = fp16(V[c][i] 2^(1-e)) with max |V[c]| = f 2^e, f in [0.5, 1) (0 rows up to
// the 128-padded size and for c >= R); vinv = 2^(e-1).
__global__ void tc_group_convert_kernel(const BMember *mem, const BChunk *chunks, int nchunks, const float *V, int R,
                                        int R_pad, const unsigned *colmax, __half *V16, int64_t v_cols, float *vinv,
                                        const int *mdone, int split) {
    const int c = blockIdx.y;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const BChunk k = chunks[ch];
        if (mdone && mdone[k.member]) continue;
        const BMember &m = mem[k.member];
        float scale = 0.0f, inv = 1.0f;
        if (c < R) {
            const float mx = __uint_as_float(colmax[(int64_t)k.member * R_pad + c]);
            int e = 0;
            if (mx > 0.0f && isfinite(mx)) {
                frexpf(mx, &e);
                scale = ldexpf(1.0f, 1 - e);
                inv = ldexpf(1.0f, e - 1);
            } else {
                scale = 1.0f;
            }
        }
        if (k.start == 0 && threadIdx.x == 0) vinv[(int64_t)k.member * R_pad + c] = inv;
        const int64_t n_pad = rup(m.n, TM);
        const float *v = V + m.vo + (int64_t)c * m.n;
        __half *out = V16 + (int64_t)c * v_cols + m.cb;
        __half *lo = split ? out + (int64_t)R_pad * v_cols : nullptr;  // low parts (split form)
        for (int r = threadIdx.x; r < kBatchChunk; r += blockDim.x) {
            const int64_t i = (int64_t)k.start + r;
            if (i >= n_pad) break;
            const float x = (c < R && i < m.n) ? v[i] * scale : 0.0f;
            const __half h = __float2half_rn(x);
            out[i] = h;
            if (lo) lo[i] = __float2half_rn(x - __half2float(h));
        }
    }
}

// Column-wise max |V| partials (grid P x R).
__global__ void tc_colmax_kernel(const float *V, int64_t ldv, int64_t n, int P, float *part, const int *done) {
    if (done && *done) return;
    const int pidx = blockIdx.x, c = blockIdx.y;
    const int64_t per = cdiv(n, P), i0 = pidx * per, i1 = min(n, i0 + per);
    float m = 0.0f;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) m = fmaxf(m, fabsf(V[(int64_t)c * ldv + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
        part[(int64_t)c * P + pidx] = t;
    }
}

// V16[c][j] = fp16(V[c][j] * 2^-e_c) for j < n, 0 up to n_pad and for c >= R; with V16lo also
// the low part fp16(V[c][j] * 2^-e_c - V16[c][j]) (the split form).
__global__ void tc_convert_kernel(const float *V, int64_t ldv, int64_t n, int64_t n_pad, int R, int P,
                                  const float *part, __half *V16, __half *V16lo, float *vinv, const int *done) {
    if (done && *done) return;
    const int c = blockIdx.y;
    float scale = 0.0f, inv = 1.0f;
    __shared__ float s_m;
    if (c < R && threadIdx.x < 32) {
        float mw = 0.0f;
        for (int q = threadIdx.x; q < P; q += 32) mw = fmaxf(mw, part[(int64_t)c * P + q]);
        for (int o = 16; o > 0; o >>= 1) mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
        if (threadIdx.x == 0) s_m = mw;
    }
    __syncthreads();
    if (c < R) {
        const float m = s_m;
        int e = 0;
        if (m > 0.0f && isfinite(m)) frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
        scale = ldexpf(1.0f, 1 - e);                  // m * scale in [1, 2)
        inv = ldexpf(1.0f, e - 1);
        if (!(m > 0.0f) || !isfinite(m)) {
            scale = 1.0f;
            inv = 1.0f;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) vinv[c] = inv;
    }
    const float *vc = V + (int64_t)c * ldv;
    if ((n & 3) == 0 && (ldv & 3) == 0 && (reinterpret_cast<uintptr_t>(V) & 15) == 0) {
        // four values per thread: one float4 load, one 8-byte store (n_pad is a multiple of 128)
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (n_pad >> 2);
             q += (int64_t)gridDim.x * blockDim.x) {
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (c < R && 4 * q < n) v = reinterpret_cast<const float4 *>(vc)[q];
            const float4 w = make_float4(v.x * scale, v.y * scale, v.z * scale, v.w * scale);
            __half2 lo = __floats2half2_rn(w.x, w.y), hi = __floats2half2_rn(w.z, w.w);
            uint2 u;
            u.x = *reinterpret_cast<uint32_t *>(&lo);
            u.y = *reinterpret_cast<uint32_t *>(&hi);
            reinterpret_cast<uint2 *>(V16 + (int64_t)c * n_pad)[q] = u;
            if (V16lo) {
                const float2 fl = __half22float2(lo), fh = __half22float2(hi);
                __half2 rl = __floats2half2_rn(w.x - fl.x, w.y - fl.y), rh = __floats2half2_rn(w.z - fh.x, w.w - fh.y);
                u.x = *reinterpret_cast<uint32_t *>(&rl);
                u.y = *reinterpret_cast<uint32_t *>(&rh);
                reinterpret_cast<uint2 *>(V16lo + (int64_t)c * n_pad)[q] = u;
            }
        }
        return;
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_pad; j += (int64_t)gridDim.x * blockDim.x) {
        float v = (c < R && j < n) ? vc[j] * scale : 0.0f;
        const __half h = __float2half_rn(v);
        V16[(int64_t)c * n_pad + j] = h;
        if (V16lo) V16lo[(int64_t)c * n_pad + j] = __float2half_rn(v - __half2float(h));
    }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

int make_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
             uint32_t box_outer) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is unavailable");
        return GP_ERR_UNSUPPORTED;
    }
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return GP_ERR_CUDA;
    }
    return GP_OK;
}

int kd_for(int d) { return (int)rup(3 * d + 4, 64); }
int rpad_for(int R) { return (int)rup(R, 16); }
}  // namespace
int tc_rhs_pad(int R) { return rpad_for(R); }
int64_t tc_cols_pad(int64_t n) { return rup(std::max<int64_t>(n, 1), TN); }
namespace {

int num_sms_tc() { return device_sm_count(); }

// The persistent schedule (split code kPersist): one CTA per SM over equal runs of
// (row tile, column tile) pairs; nseg = the most row segments one CTA can meet.
void persist_geom(int64_t row_tiles, int64_t col_tiles, int *G, int *nseg) {
    const int64_t T = row_tiles * col_tiles;
    const int64_t g = std::max<int64_t>(1, std::min<int64_t>(std::min(num_sms_tc(), kPersistMaxGrid), T));
    *G = (int)g;
    *nseg = (int)(cdiv(cdiv(T, g), col_tiles) + 1);
}

// Column splits per row tile: minimises (waves of CTAs) x (tiles per CTA + a fixed per-CTA
// cost of about four tiles: tensor-memory allocation, first loads, epilogue); every split
// owns at least one tile.  Few row tiles (a stochastic-gradient row panel) get many splits.
int pick_uniform_split(int64_t row_tiles, int64_t col_tiles, int64_t *cost_out) {
    const int64_t sms = num_sms_tc();
    const int64_t smax = std::min<int64_t>(256, std::max<int64_t>(1, col_tiles));
    int best = 1;
    int64_t best_cost = INT64_MAX;
    for (int64_t s = 1; s <= smax; ++s) {
        if (s > 1 && cdiv(col_tiles, s) * (s - 1) >= col_tiles) continue;
        const int64_t cost = cdiv(row_tiles * s, sms) * (cdiv(col_tiles, s) + 4) + (s > 1 ? 1 : 0);
        if (cost < best_cost) {
            best_cost = cost;
            best = (int)s;
        }
    }
    if (cost_out) *cost_out = best_cost;
    return best;
}

// The product's schedule: the best uniform split, or the persistent one when the model
// prices it lower: no partial last wave and one start-up per SM, against about two tiles per
// extra row segment (row-operand reload, accumulator read-out), the straddling rows'
// reduction, and a tile period about 2% longer than the uniform split's (measured at
// n = 32768 to 131072).
int pick_split(int64_t row_tiles, int64_t col_tiles) {
    int64_t ucost = 0;
    const int best = pick_uniform_split(row_tiles, col_tiles, &ucost);
    int G = 0, sg = 0;
    persist_geom(row_tiles, col_tiles, &G, &sg);
    const int64_t pcost = (cdiv(row_tiles * col_tiles, G) * 102 + 99) / 100 + 4 + 2 * (int64_t)(sg - 1) + 1;
    return pcost < ucost ? kPersist : best;
}

// Floats of partial sums a product with this split code needs.
size_t partial_floats(int split, int64_t n1, int R, int64_t row_tiles, int64_t col_tiles) {
    if (split == kPersist) {
        int G = 0, sg = 0;
        persist_geom(row_tiles, col_tiles, &G, &sg);
        return (size_t)G * 2 * R * TM;  // two slots per CTA
    }
    return split > 1 ? (size_t)split * R * n1 : 0;
}

// Choices of the autotuner (gp_autotune_mvm, gp_autotune_grad), keyed by kernel and shape:
//   product  : (0, R_pad, row tiles, column tiles) -> split code (kPersist or column splits)
//   gradient : (1, KD, KM, row tiles, symmetric)   -> tile pairs per item (symmetric sweep) or
//                                                     column splits per row tile
// They replace the built-in rules wherever the caller's workspace holds what they need.  The
// table can be written to and read from a text file (gp_autotune_save / gp_autotune_load), and
// is read at first use from the file named by GP_AUTOTUNE_CACHE (and written back to it after
// every tuning call) when that variable is set.
using TuneKey = std::array<int64_t, 5>;
struct TuneTable {
    std::mutex mu;
    std::map<TuneKey, int64_t> best;
    bool env_loaded = false;
};
TuneTable &tune_table() {
    static TuneTable t;
    return t;
}
thread_local int g_force_split = 0;      // set by the autotuner while it times one candidate
thread_local int64_t g_force_grad = 0;   // likewise for the gradient kernel's work split

// Device identity written into (and checked against) a cache file.
std::string tune_device_id() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return std::string("unknown");
    }
    std::string name(prop.name);
    for (char &ch : name)
        if (ch == ' ') ch = '_';
    return name + "_sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "_x" +
           std::to_string(prop.multiProcessorCount);
}

// Reads a cache file into t (lock held).  Returns GP_OK, or GP_ERR_INVALID_ARG for a missing
// or unreadable file, another device's file or a malformed line (the table is then unchanged).
int tune_read_locked(TuneTable &t, const char *path) {
    FILE *f = std::fopen(path, "r");
    if (!f) {
        set_error("autotune cache %s cannot be opened", path);
        return GP_ERR_INVALID_ARG;
    }
    char head[64] = {0}, dev[256] = {0};
    int ver = 0;
    if (std::fscanf(f, "%63s %d %255s", head, &ver, dev) != 3 || std::string(head) != "gp_gb300_autotune" ||
        ver != 1) {
        std::fclose(f);
        set_error("autotune cache %s: not a version-1 cache file", path);
        return GP_ERR_INVALID_ARG;
    }
    if (tune_device_id() != dev) {
        std::fclose(f);
        set_error("autotune cache %s was written on another device (%s)", path, dev);
        return GP_ERR_INVALID_ARG;
    }
    std::map<TuneKey, int64_t> rd;
    long long k0, k1, k2, k3, k4, v;
    int got;
    while ((got = std::fscanf(f, "%lld %lld %lld %lld %lld %lld", &k0, &k1, &k2, &k3, &k4, &v)) == 6)
        rd[TuneKey{k0, k1, k2, k3, k4}] = v;
    std::fclose(f);
    if (got != EOF) {
        set_error("autotune cache %s: malformed entry", path);
        return GP_ERR_INVALID_ARG;
    }
    for (const auto &e : rd) t.best[e.first] = e.second;
    return GP_OK;
}

int tune_write_locked(const TuneTable &t, const char *path) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) {
        set_error("autotune cache %s cannot be written", path);
        return GP_ERR_INVALID_ARG;
    }
    std::fprintf(f, "gp_gb300_autotune 1 %s\n", tune_device_id().c_str());
    for (const auto &e : t.best)
        std::fprintf(f, "%lld %lld %lld %lld %lld %lld\n", (long long)e.first[0], (long long)e.first[1],
                     (long long)e.first[2], (long long)e.first[3], (long long)e.first[4], (long long)e.second);
    const bool ok = std::fclose(f) == 0 && std::rename(tmp.c_str(), path) == 0;
    if (!ok) {
        set_error("autotune cache %s cannot be written", path);
        return GP_ERR_INVALID_ARG;
    }
    return GP_OK;
}

// Reads GP_AUTOTUNE_CACHE once per process (lock held); a missing or unusable file leaves the
// built-in rules in place.
void tune_env_load_locked(TuneTable &t) {
    if (t.env_loaded) return;
    t.env_loaded = true;
    const char *path = std::getenv("GP_AUTOTUNE_CACHE");
    if (path && *path && tune_read_locked(t, path) != GP_OK) clear_error();
}

// The entry for key, or 0.
int64_t tune_get(const TuneKey &key) {
    TuneTable &t = tune_table();
    std::lock_guard<std::mutex> g(t.mu);
    tune_env_load_locked(t);
    auto it = t.best.find(key);
    return it == t.best.end() ? 0 : it->second;
}

int tune_put(const TuneKey &key, int64_t v) {
    tune_get(key);  // the environment's cache first, so that writing it back keeps its entries
    TuneTable &t = tune_table();
    std::lock_guard<std::mutex> g(t.mu);
    t.best[key] = v;
    const char *path = std::getenv("GP_AUTOTUNE_CACHE");
    if (path && *path) return tune_write_locked(t, path);
    return GP_OK;
}

int tuned_split(int R_pad, int64_t row_tiles, int64_t col_tiles) {
    return (int)tune_get(TuneKey{0, R_pad, row_tiles, col_tiles, 0});
}

// The split a product of this shape uses: forced (autotuner), tuned, or the cost model.
int split_for(int R_pad, int64_t row_tiles, int64_t col_tiles) {
    if (g_force_split != 0) return g_force_split;
    const int t = tuned_split(R_pad, row_tiles, col_tiles);
    return t != 0 ? t : pick_split(row_tiles, col_tiles);
}

// Ring depths of the product kernel: up to 4 V slots (GEMM2 runs about two tiles behind
// GEMM1), the rest of shared memory for PB slots (at most MAX_RING).  The split form's V slot
// holds the high and the low parts (twice the bytes).
void rings_for(int KD, int R_pad, int *npb, int *nv, bool split = false) {
    const size_t a = (size_t)TM * KD * 2, b = (size_t)TN * KD * 2, v = (split ? 4 : 2) * (size_t)R_pad * 128;
    const size_t budget = kMaxDynSmem - 4096 - a;
    int nvv = 4;
    while (nvv > 2 && nvv * v + 3 * b > budget) --nvv;
    size_t left = budget > nvv * v ? budget - nvv * v : 0;
    *nv = nvv;
    *npb = (int)std::min<size_t>(MAX_RING, left / b);
}

size_t smem_for(int KD, int R_pad, int npb, int nv, bool split = false) {
    return 1024 + (size_t)TM * KD * 2 + (size_t)npb * TN * KD * 2 + (size_t)nv * (split ? 4 : 2) * R_pad * 128 + 512;
}

// Right-hand sides per pass of the split form for a contraction width KD: the largest multiple
// of 16 (at most kMaxRhsPerPass) whose rings fit shared memory.
int split_rhs_per_pass(int KD) {
    for (int r = kSplitMaxRpad; r >= 16; r -= 16) {
        int npb = 0, nv = 0;
        rings_for(KD, r, &npb, &nv, true);
        if (npb >= 2 && nv >= 2) return r;
    }
    return 0;
}

template <int KIND, int KAT, bool PERSIST, bool SPLIT>
int launch_mvm_kernel(dim3 grid, size_t smem, const CUtensorMap &mA, const CUtensorMap &mB, const CUtensorMap &mV,
                      const KParams &kp, cudaStream_t st) {
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<KIND, KAT, PERSIST, SPLIT>));
    tc_mvm_kernel<KIND, KAT, PERSIST, SPLIT><<<grid, MVM_THREADS, smem, st>>>(mA, mB, mV, kp);
    return GP_OK;
}

template <int KIND, int KAT>
int launch_mvm_kernel(dim3 grid, size_t smem, const CUtensorMap &mA, const CUtensorMap &mB, const CUtensorMap &mV,
                      const KParams &kp, bool split, cudaStream_t st) {
    if (split) {  // the split form runs a single segment per CTA (no persistent schedule)
        if (kp.persist) {
            set_error("internal: the split product has no persistent schedule");
            return GP_ERR_UNSUPPORTED;
        }
        return launch_mvm_kernel<KIND, KAT, false, true>(grid, smem, mA, mB, mV, kp, st);
    }
    return kp.persist ? launch_mvm_kernel<KIND, KAT, true, false>(grid, smem, mA, mB, mV, kp, st)
                      : launch_mvm_kernel<KIND, KAT, false, false>(grid, smem, mA, mB, mV, kp, st);
}

}  // namespace

int tc_make_map16(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                  uint32_t box_outer) {
    return make_map(m, base, inner, outer, box_inner, box_outer);
}

// The status word's device address, looked up once per device (a symbol's address differs
// between devices) under a lock.
int *tc_timeout_word() {
    static std::mutex mu;
    static std::map<int, int *> words;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> g(mu);
    auto it = words.find(dev);
    if (it != words.end()) return it->second;
    void *a = nullptr;
    if (cudaGetSymbolAddress(&a, g_tc_timeout) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    words[dev] = static_cast<int *>(a);
    return static_cast<int *>(a);
}

int tc_timeout_status(cudaStream_t st) {
    int *w = tc_timeout_word();
    if (!w) return GP_OK;
    int h = 0;
    GP_TRY_CUDA(cudaMemcpyAsync(&h, w, sizeof(int), cudaMemcpyDeviceToHost, st));
    GP_TRY_CUDA(cudaStreamSynchronize(st));
    if (h) {
        GP_TRY_CUDA(cudaMemsetAsync(w, 0, sizeof(int), st));
        GP_TRY_CUDA(cudaStreamSynchronize(st));
        set_error("a bounded wait in a tensor-core kernel gave up (its results are not valid)");
        return GP_ERR_TIMEOUT;
    }
    return GP_OK;
}

namespace {
// A wait that nothing completes, bounded by `limit` cycles: exercises the time-out path.
__global__ void tc_timeout_probe_kernel(long long limit, int *word) {
    __shared__ uint64_t bar;
    __shared__ int err;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait_for(&bar, 0, &err, limit);
    __syncthreads();
    if (threadIdx.x == 0 && !ok && word) atomicExch(word, 1);
}
}  // namespace

int tc_timeout_probe(long long limit, cudaStream_t st) {
    tc_timeout_probe_kernel<<<1, 32, 0, st>>>(limit, tc_timeout_word());
    return check_launch("tc_timeout_probe_kernel");
}

bool tc_available() {
    static std::mutex mu;
    static std::map<int, bool> ok;
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> g(mu);
    auto it = ok.find(dev);
    if (it != ok.end()) return it->second;
    bool v = false;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) == cudaSuccess)
        v = (major == 10 && minor == 3) && encode_fn() != nullptr;
    else
        cudaGetLastError();
    ok[dev] = v;
    return v;
}

// Buffer of a prepared pair: PA (n1_pad x KD), PB (n2_pad x KD), bound, dscale.
size_t tc_points_bytes(int64_t n, int d) {
    Carver c(nullptr);
    c.take<__half>((size_t)rup(std::max<int64_t>(n, 1), TM) * kd_for(d));
    c.take<__half>((size_t)rup(std::max<int64_t>(n, 1), TN) * kd_for(d));
    c.take<unsigned int>(1);
    c.take<float>(1);
    return c.bytes();
}

int tc_prepare_points(const KP<float> &kp, const float *X, int64_t n, void *buf, TcPoints *out, cudaStream_t st) {
    return tc_prepare_points_dev(kp, X, n, buf, out, nullptr, st);
}

// Same, with the length-scales read from device memory when inv_dev is set.
int tc_prepare_points_dev(const KP<float> &kp, const float *X, int64_t n, void *buf, TcPoints *out,
                          const float *inv_dev, cudaStream_t st) {
    const int KD = kd_for(kp.d);
    const int64_t n_pad = rup(std::max<int64_t>(n, 1), TM);
    Carver c(buf);
    __half *PA = c.take<__half>((size_t)n_pad * KD);
    __half *PB = c.take<__half>((size_t)n_pad * KD);
    unsigned int *bound = c.take<unsigned int>(1);
    float *dscale = c.take<float>(1);
    const float cf = (kp.kind == GP_RBF) ? -0.5f * kLog2e : 3.0f * kLog2e * kLog2e;
    GP_TRY_CUDA(cudaMemsetAsync(bound, 0, sizeof(unsigned int), st));
    const unsigned nb = (unsigned)std::min<int64_t>(cdiv(n_pad, 256), 1024);
    tc_bound_kernel<<<nb, 256, 0, st>>>(kp, cf, X, n, bound, inv_dev);
    tc_operands_kernel<<<operand_blocks(n_pad), 256, 0, st>>>(kp, cf, X, n, n_pad, KD, bound, PA, PB, dscale, inv_dev);
    GP_TRY(check_launch("tc operand preparation", 2));
    out->PA = PA;
    out->PB = PB;
    out->n = n;
    out->n_pad = n_pad;
    out->KD = KD;
    out->dscale = dscale;
    out->bound = bound;
    return GP_OK;
}

int tc_prepare_pair(const KP<float> &kp, const float *X1, int64_t n1, const float *X2, int64_t n2, void *buf1,
                    void *buf2, TcPoints *rows, TcPoints *cols, cudaStream_t st) {
    // one shared scale for both point sets: bound over the union
    const int KD = kd_for(kp.d);
    const int64_t p1 = rup(std::max<int64_t>(n1, 1), TM), p2 = rup(std::max<int64_t>(n2, 1), TM);
    Carver c1(buf1), c2(buf2);
    __half *PA = c1.take<__half>((size_t)p1 * KD);
    c1.take<__half>((size_t)p1 * KD);
    unsigned int *bound = c1.take<unsigned int>(1);
    float *dscale = c1.take<float>(1);
    c2.take<__half>((size_t)p2 * KD);
    __half *PB = c2.take<__half>((size_t)p2 * KD);
    const float cf = (kp.kind == GP_RBF) ? -0.5f * kLog2e : 3.0f * kLog2e * kLog2e;
    GP_TRY_CUDA(cudaMemsetAsync(bound, 0, sizeof(unsigned int), st));
    tc_bound_kernel<<<(unsigned)std::min<int64_t>(cdiv(p1, 256), 1024), 256, 0, st>>>(kp, cf, X1, n1, bound,
                                                                                       nullptr);
    tc_bound_kernel<<<(unsigned)std::min<int64_t>(cdiv(p2, 256), 1024), 256, 0, st>>>(kp, cf, X2, n2, bound,
                                                                                       nullptr);
    tc_operands_kernel<<<operand_blocks(p1), 256, 0, st>>>(
        kp, cf, X1, n1, p1, KD, bound, PA, nullptr, dscale, nullptr);
    tc_operands_kernel<<<operand_blocks(p2), 256, 0, st>>>(
        kp, cf, X2, n2, p2, KD, bound, nullptr, PB, nullptr, nullptr);
    GP_TRY(check_launch("tc pair preparation", 4));
    *rows = TcPoints{PA, nullptr, n1, p1, KD, dscale, bound};
    *cols = TcPoints{nullptr, PB, n2, p2, KD, dscale, bound};
    return GP_OK;
}

int tc_prepare_rows(const KP<float> &kp, const float *X1, int64_t n1, const TcPoints &like, void *buf, TcPoints *out,
                    cudaStream_t st) {
    const int KD = like.KD;
    const int64_t p1 = rup(std::max<int64_t>(n1, 1), TM);
    Carver c(buf);
    __half *PA = c.take<__half>((size_t)p1 * KD);
    const float cf = (kp.kind == GP_RBF) ? -0.5f * kLog2e : 3.0f * kLog2e * kLog2e;
    // the bound of the prepared superset fixes the same power-of-two scale
    tc_operands_kernel<<<operand_blocks(p1), 256, 0, st>>>(
        kp, cf, X1, n1, p1, KD, like.bound, PA, nullptr, nullptr, nullptr);
    GP_TRY(check_launch("tc row preparation"));
    *out = TcPoints{PA, nullptr, n1, p1, KD, like.dscale, like.bound};
    return GP_OK;
}

// Generation of a persistent launch (40 bits): distinct for every launch of the process (an odd
// multiple mod 2^40 of a running count is a bijection), never 0, and spread over the 40 bits so
// that stale memory rarely matches it.
unsigned long long next_generation() {
    static std::atomic<unsigned long long> count{0};
    constexpr unsigned long long kMask = (1ull << 40) - 1ull;
    unsigned long long g = 0;
    while (g == 0) g = ((count.fetch_add(1, std::memory_order_relaxed) + 1ull) * 0x9E3779B97F4Bull) & kMask;
    return g;
}

size_t tc_mvm_workspace_for(int64_t n1, int64_t p2, int R, int nsplit) {
    const int R_pad = rpad_for(std::min(R, kMaxRhsPerPass));
    Carver c(nullptr);
    c.take<__half>((size_t)2 * R_pad * p2);  // V16: high parts, then the split form's low parts
    c.take<float>(256);
    c.take<float>((size_t)std::min(R, kMaxRhsPerPass) * 64);
    c.take<int>(1);
    c.take<unsigned long long>((size_t)cdiv(std::max<int64_t>(n1, 1), TM) * 8);
    const size_t pf = partial_floats(nsplit, n1, std::min(R, kMaxRhsPerPass), cdiv(std::max<int64_t>(n1, 1), TM),
                                     cdiv(p2, TN));
    if (pf > 0) c.take<float>(pf);
    return c.bytes();
}

size_t tc_mvm_workspace(int64_t n1, int64_t n2, int R) {
    const int64_t p2 = rup(std::max<int64_t>(n2, 1), TN);
    const int R_pad = rpad_for(std::min(R, kMaxRhsPerPass));
    const int64_t row_tiles = cdiv(std::max<int64_t>(n1, 1), TM), col_tiles = cdiv(p2, TN);
    // room for the partial sums of both the tuned and the model's choice
    const int s1 = split_for(R_pad, row_tiles, col_tiles), s2 = pick_split(row_tiles, col_tiles);
    const int s3 = pick_uniform_split(row_tiles, col_tiles, nullptr);  // the split form's schedule
    const size_t pf = std::max(std::max(partial_floats(s1, n1, R, row_tiles, col_tiles),
                                        partial_floats(s2, n1, R, row_tiles, col_tiles)),
                               partial_floats(s3, n1, std::min(R, kSplitMaxRpad), row_tiles, col_tiles));
    Carver c(nullptr);
    c.take<__half>((size_t)2 * R_pad * p2);        // V16 (high parts; low parts of the split form)
    c.take<float>(256);                            // vinv
    c.take<float>((size_t)R * 64);                 // column max partials
    c.take<int>(1);                                // error flag
    c.take<unsigned long long>((size_t)row_tiles * 8);  // shared row tiles' arrival counters
    if (pf > 0) c.take<float>(pf);                 // partial sums
    return c.bytes();
}

int tc_mvm(const TcMvmArgs &a, void *ws, size_t ws_bytes, cudaStream_t st) {
    // right-hand sides per pass: the Y accumulator's share of tensor memory; for the split form
    // also what its doubled V slots leave of shared memory
    const int per_pass = a.split ? std::min(kMaxRhsPerPass, split_rhs_per_pass(a.rows.KD)) : kMaxRhsPerPass;
    if (per_pass < 1) {
        set_error("split tensor-core product: tile does not fit shared memory (KD=%d)", a.rows.KD);
        return GP_ERR_UNSUPPORTED;
    }
    if (a.dot_parts) *a.dot_parts = 0;
    if (a.R > per_pass) {
        // wide blocks of right-hand sides: per_pass at a time
        for (int c0 = 0; c0 < a.R; c0 += per_pass) {
            TcMvmArgs b = a;
            b.R = std::min(per_pass, a.R - c0);
            b.V16pre = nullptr;  // a caller's converted operand covers all columns at once
            b.dotpart = nullptr;  // d^T y partials only for a single pass
            b.dot_parts = nullptr;
            b.V = a.V + (int64_t)c0 * a.ldv;
            b.Y = a.Y + (int64_t)c0 * a.ldy;
            b.Vd = a.Vd ? a.Vd + (int64_t)c0 * a.ldvd : nullptr;
            GP_TRY(tc_mvm(b, ws, ws_bytes, st));
        }
        return GP_OK;
    }
    const int64_t n1 = a.rows.n, n2 = a.ncols > 0 ? a.ncols : a.cols.n;
    if (n1 == 0 || a.R == 0) return GP_OK;
    const int KD = a.rows.KD;
    const int R_pad = rpad_for(a.R);
    const int64_t p2 = rup(std::max<int64_t>(n2, 1), TN);
    const int64_t row_tiles = cdiv(n1, TM), col_tiles = cdiv(p2, TN);
    // the split form takes column splits only (its group read-out has one segment per CTA)
    int nsplit = a.split ? pick_uniform_split(row_tiles, col_tiles, nullptr) : split_for(R_pad, row_tiles, col_tiles);
    {
        // a tuned split whose partial sums do not fit the caller's workspace falls back to
        // the model's choice
        Carver probe(nullptr);
        probe.take<__half>((size_t)2 * R_pad * p2);
        probe.take<float>(256);
        probe.take<float>((size_t)a.R * 64);
        probe.take<int>(1);
        probe.take<unsigned long long>((size_t)row_tiles * 8);
        const size_t pf = partial_floats(nsplit, n1, a.R, row_tiles, col_tiles);
        if (pf > 0) probe.take<float>(pf);
        if (probe.bytes() > ws_bytes && g_force_split == 0) nsplit = a.split ? 1 : pick_split(row_tiles, col_tiles);
    }
    const bool persist = (nsplit == kPersist);
    int pgrid = 0, pseg = 0;
    if (persist) persist_geom(row_tiles, col_tiles, &pgrid, &pseg);
    const size_t pfl = partial_floats(nsplit, n1, a.R, row_tiles, col_tiles);
    Carver c(ws);
    __half *V16 = c.take<__half>((size_t)2 * R_pad * p2);  // rows [0, R_pad): high; [R_pad, 2 R_pad): low
    float *vinv = c.take<float>(256);
    float *cm = c.take<float>((size_t)a.R * 64);
    c.take<int>(1);  // (kept for the workspace layout)
    unsigned long long *pcnt = c.take<unsigned long long>((size_t)row_tiles * 8);
    int *err = tc_timeout_word();
    float *partial = pfl > 0 ? c.take<float>(pfl) : nullptr;
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    const bool pre = a.V16pre != nullptr && !a.split;  // operand converted by the caller
    if (pre) {
        V16 = static_cast<__half *>(const_cast<void *>(a.V16pre));
        vinv = const_cast<float *>(a.vinv_pre);
    } else {
        const int P = (int)std::min<int64_t>(64, std::max<int64_t>(1, cdiv(n2, 4096)));
        tc_colmax_kernel<<<dim3(P, a.R), 256, 0, st>>>(a.V, a.ldv, n2, P, cm, a.done);
        tc_convert_kernel<<<dim3((unsigned)std::min<int64_t>(cdiv(p2, 1024), 256), R_pad), 256, 0, st>>>(
            a.V, a.ldv, n2, p2, a.R, P, cm, V16, a.split ? V16 + (size_t)R_pad * p2 : nullptr, vinv, a.done);
        GP_TRY(check_launch("tc rhs conversion", 2));
    }

    CUtensorMap mA, mB, mV;
    GP_TRY(make_map(&mA, a.rows.PA, KD, a.rows.n_pad, 64, TM));
    GP_TRY(make_map(&mB, a.cols.PB, KD, a.cols.n_pad, 64, TN));
    GP_TRY(make_map(&mV, V16, p2, a.split ? 2 * R_pad : R_pad, 64, R_pad));
    int npb = 0, nv = 0;
    rings_for(KD, R_pad, &npb, &nv, a.split);
    if (npb < 2 || nv < 2) {
        set_error("tensor-core tile does not fit shared memory (d=%d, R=%d)", (KD - 4) / 3, a.R);
        return GP_ERR_UNSUPPORTED;
    }
    KParams kp{};
    kp.R = a.R;
    kp.R_pad = R_pad;
    kp.KD = KD;
    kp.npb = npb;
    kp.nv = nv;
    kp.n1 = n1;
    kp.col_tiles = col_tiles;
    kp.nsplit = persist ? 1 : nsplit;
    kp.persist = persist ? 1 : 0;
    kp.ptotal = row_tiles * col_tiles;
    kp.pgrid = pgrid;
    kp.sf2 = a.sf2;
    kp.alpha = a.alpha;
    kp.beta = a.beta;
    kp.diag_coef = a.diag_coef;
    kp.vinv = vinv;
    kp.dscale = a.rows.dscale;
    kp.Vd = a.Vd;
    kp.ldvd = a.ldvd;
    kp.drow0 = a.drow0;
    kp.ndiag = a.ndiag;
    kp.Y = a.Y;
    kp.ldy = a.ldy;
    kp.partial = partial;
    kp.done = a.done;
    kp.err = err;
    kp.col0_dev = a.col0_dev;
    kp.diag_from_col0 = a.diag_from_col0;
    kp.ncols_total = a.cols.n;
    if (persist) {
        kp.pcnt = pcnt;
        kp.pgen = next_generation();
        if (a.dotpart) {
            kp.dotv = a.dotv;
            kp.lddv = a.lddv;
            kp.dotpart = a.dotpart;
        }
    }
    if (a.dot_parts) *a.dot_parts = (persist && a.dotpart) ? pgrid : 0;
    const size_t smem = smem_for(KD, R_pad, npb, nv, a.split);
    dim3 grid = persist ? dim3((unsigned)pgrid, 1) : dim3((unsigned)row_tiles, (unsigned)nsplit);
    const int kat = KD / 64;
    if (kat > 3) {
        set_error("tensor-core product supports d <= 62 (got KD=%d)", KD);
        return GP_ERR_UNSUPPORTED;
    }
    prof_begin(st);
    if (a.kind == GP_RBF) {
        if (kat == 1) GP_TRY(launch_mvm_kernel<GP_RBF, 1>(grid, smem, mA, mB, mV, kp, a.split != 0, st));
        else if (kat == 2) GP_TRY(launch_mvm_kernel<GP_RBF, 2>(grid, smem, mA, mB, mV, kp, a.split != 0, st));
        else GP_TRY(launch_mvm_kernel<GP_RBF, 3>(grid, smem, mA, mB, mV, kp, a.split != 0, st));
    } else {
        if (kat == 1) GP_TRY(launch_mvm_kernel<GP_MATERN32, 1>(grid, smem, mA, mB, mV, kp, a.split != 0, st));
        else if (kat == 2) GP_TRY(launch_mvm_kernel<GP_MATERN32, 2>(grid, smem, mA, mB, mV, kp, a.split != 0, st));
        else GP_TRY(launch_mvm_kernel<GP_MATERN32, 3>(grid, smem, mA, mB, mV, kp, a.split != 0, st));
    }
    prof_end(st);
    GP_TRY(check_launch("tc_mvm_kernel"));
    if (persist) {
        // the shared row tiles are finished inside the kernel
    } else if (nsplit > 1) {
        tc_reduce_kernel<<<dim3((unsigned)cdiv(n1, 256), a.R), 256, 0, st>>>(kp);
        GP_TRY(check_launch("tc_reduce_kernel"));
    }
    return GP_OK;
}

// Times the product H V (a.rows == a.cols) for a ladder of split counts and records the
// fastest for its shape.  Synchronises `st`; not for use inside a stream capture.
int tc_autotune(const TcMvmArgs &a, int reps, void *ws, size_t ws_bytes, cudaStream_t st, int *best_split,
                double *best_ms) {
    const int64_t n1 = a.rows.n;
    const int64_t p2 = rup(std::max<int64_t>(a.cols.n, 1), TN);
    const int R_pad = rpad_for(std::min(a.R, kMaxRhsPerPass));
    const int64_t row_tiles = cdiv(std::max<int64_t>(n1, 1), TM), col_tiles = cdiv(p2, TN);
    static const int ladder[] = {kPersist, 1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 16, 24, 32, 48, 64, 96, 128};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GP_TRY_CUDA(cudaEventCreate(&e0));
    GP_TRY_CUDA(cudaEventCreate(&e1));
    int best = 0;
    double best_t = 1e300;
    int rc = GP_OK;
    for (int s : ladder) {
        if (s != kPersist && (s > col_tiles || (s > 1 && cdiv(col_tiles, s) * (s - 1) >= col_tiles))) continue;
        if (tc_mvm_workspace_for(n1, p2, a.R, s) > ws_bytes) continue;
        g_force_split = s;
        double t_min = 1e300;
        for (int r = 0; r <= reps && rc == GP_OK; ++r) {  // the first run is a warm-up
            if (cudaEventRecord(e0, st) != cudaSuccess) rc = GP_ERR_CUDA;
            if (rc == GP_OK) rc = tc_mvm(a, ws, ws_bytes, st);
            if (rc == GP_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = GP_ERR_CUDA;
            if (rc == GP_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = GP_ERR_CUDA;
            float ms = 0.0f;
            if (rc == GP_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = GP_ERR_CUDA;
            if (rc == GP_OK && r > 0) t_min = std::min(t_min, (double)ms);
        }
        g_force_split = 0;
        if (rc != GP_OK) break;
        if (t_min < best_t) {
            best_t = t_min;
            best = s;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GP_OK) {
        set_error("autotune: a timed product failed");
        return rc;
    }
    if (best == 0) {
        set_error("autotune: the workspace holds no candidate");
        return GP_ERR_WORKSPACE;
    }
    GP_TRY(tune_put(TuneKey{0, R_pad, row_tiles, col_tiles, 0}, best));
    *best_split = best;
    *best_ms = best_t;
    return GP_OK;
}

size_t tc_autotune_workspace(int64_t n, int R) {
    const int64_t p2 = rup(std::max<int64_t>(n, 1), TN);
    const int64_t col_tiles = p2 / TN;
    return std::max(tc_mvm_workspace_for(n, p2, R, (int)std::min<int64_t>(128, col_tiles)),
                    tc_mvm_workspace_for(n, p2, R, kPersist));
}

void tc_autotune_reset() {
    TuneTable &t = tune_table();
    std::lock_guard<std::mutex> g(t.mu);
    t.best.clear();
    t.env_loaded = true;  // a reset table stays empty (the environment's cache is not re-read)
}

int tc_autotune_save(const char *path) {
    TuneTable &t = tune_table();
    std::lock_guard<std::mutex> g(t.mu);
    return tune_write_locked(t, path);
}

int tc_autotune_load(const char *path) {
    TuneTable &t = tune_table();
    std::lock_guard<std::mutex> g(t.mu);
    t.env_loaded = true;
    return tune_read_locked(t, path);
}

int64_t tc_autotune_count() {
    TuneTable &t = tune_table();
    std::lock_guard<std::mutex> g(t.mu);
    tune_env_load_locked(t);
    return (int64_t)t.best.size();
}

// Grouped product over a batch of independent GPs: one CTA per work item (128 rows of a
// member against a run of its own column tiles), items ordered longest first so the
// block scheduler fills the SMs like a longest-processing-time list schedule.
int tc_group_setup() {
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_RBF, 1, false, false>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_RBF, 2, false, false>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_RBF, 3, false, false>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_MATERN32, 1, false, false>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_MATERN32, 2, false, false>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_MATERN32, 3, false, false>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_RBF, 1, false, true>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_RBF, 2, false, true>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_RBF, 3, false, true>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_MATERN32, 1, false, true>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_MATERN32, 2, false, true>));
    GP_TRY(ensure_max_dyn_smem((const void *)tc_mvm_kernel<GP_MATERN32, 3, false, true>));
    return GP_OK;
}

bool tc_split_fits_rpad(int R_pad) { return R_pad <= kSplitMaxRpad; }

int tc_group_mvm(const TcGroupArgs &a, cudaStream_t st) {
    if (a.nitems == 0) return GP_OK;
    if (a.split && a.R_pad > kSplitMaxRpad) {
        set_error("split batched product supports at most %d right-hand sides", kSplitMaxRpad);
        return GP_ERR_UNSUPPORTED;
    }
    if (a.R > kMaxRhsPerPass) {
        set_error("batched product supports at most %d right-hand sides", kMaxRhsPerPass);
        return GP_ERR_UNSUPPORTED;
    }
    const int kat = a.KD / 64;
    if (kat < 1 || kat > 3) {
        set_error("batched product supports d <= 62 (got KD=%d)", a.KD);
        return GP_ERR_UNSUPPORTED;
    }
    GP_TRY(tc_group_setup());
    CUtensorMap mA, mB, mV;
    GP_TRY(make_map(&mA, a.PA, a.KD, a.class_rows, 64, TM));
    GP_TRY(make_map(&mB, a.PB, a.KD, a.class_rows, 64, TN));
    GP_TRY(make_map(&mV, a.V16, a.v_cols, a.split ? 2 * a.R_pad : a.R_pad, 64, a.R_pad));
    int npb = 0, nv = 0;
    rings_for(a.KD, a.R_pad, &npb, &nv, a.split != 0);
    if (npb < 2 || nv < 2) {
        set_error("tensor-core tile does not fit shared memory (KD=%d, R=%d)", a.KD, a.R);
        return GP_ERR_UNSUPPORTED;
    }
    KParams kp{};
    kp.R = a.R;
    kp.R_pad = a.R_pad;
    kp.KD = a.KD;
    kp.npb = npb;
    kp.nv = nv;
    kp.nsplit = 1;
    kp.alpha = 1.0f;
    kp.beta = 0.0f;
    kp.diag_coef = a.diag;
    kp.vinv = a.vinv;
    kp.Vd = a.Vd;
    kp.Y = a.Y;
    kp.err = a.err;
    kp.items = a.items;
    kp.members = a.members;
    kp.mdone = a.mdone;
    const size_t smem = smem_for(a.KD, a.R_pad, npb, nv, a.split != 0);
    dim3 grid((unsigned)a.nitems, 1);
    const bool sp = a.split != 0;
    prof_begin(st);
    if (a.kind == GP_RBF) {
        if (kat == 1) GP_TRY(launch_mvm_kernel<GP_RBF, 1>(grid, smem, mA, mB, mV, kp, sp, st));
        else if (kat == 2) GP_TRY(launch_mvm_kernel<GP_RBF, 2>(grid, smem, mA, mB, mV, kp, sp, st));
        else GP_TRY(launch_mvm_kernel<GP_RBF, 3>(grid, smem, mA, mB, mV, kp, sp, st));
    } else {
        if (kat == 1) GP_TRY(launch_mvm_kernel<GP_MATERN32, 1>(grid, smem, mA, mB, mV, kp, sp, st));
        else if (kat == 2) GP_TRY(launch_mvm_kernel<GP_MATERN32, 2>(grid, smem, mA, mB, mV, kp, sp, st));
        else GP_TRY(launch_mvm_kernel<GP_MATERN32, 3>(grid, smem, mA, mB, mV, kp, sp, st));
    }
    prof_end(st);
    return check_launch("tc_mvm_kernel (batched)");
}

int tc_group_prepare(int kind, BMember *members, int G, const BChunk *chunks, int nchunks, const float *X,
                     void *const *PA, void *const *PB, const int *KD, cudaStream_t st) {
    (void)G;
    if (nchunks == 0) return GP_OK;
    const float cf = (kind == GP_RBF) ? -0.5f * kLog2e : 3.0f * kLog2e * kLog2e;
    const unsigned nb = (unsigned)std::min(nchunks, 8 * num_sms_tc());
    tc_group_bound_kernel<<<nb, 256, 0, st>>>(members, chunks, nchunks, X, cf);
    GroupOut o{};
    for (int c = 0; c < 3; ++c) {
        o.PA[c] = static_cast<__half *>(PA[c]);
        o.PB[c] = static_cast<__half *>(PB[c]);
        o.KD[c] = KD[c];
    }
    tc_group_operands_kernel<<<nb, 256, 0, st>>>(members, chunks, nchunks, X, cf, o);
    return check_launch("batched operand preparation", 2);
}

int tc_group_convert(const BMember *members, int G, const BChunk *chunks, int nchunks, const float *V, int R,
                     int R_pad, unsigned *colmax, void *V16, int64_t v_cols, float *vinv, const int *mdone,
                     cudaStream_t st, bool split) {
    if (nchunks == 0) return GP_OK;
    GP_TRY_CUDA(cudaMemsetAsync(colmax, 0, sizeof(unsigned) * (size_t)G * R_pad, st));
    const unsigned nb = (unsigned)std::min(nchunks, 4 * num_sms_tc());
    tc_group_colmax_kernel<<<dim3(nb, R), 256, 0, st>>>(members, chunks, nchunks, V, R, R_pad, colmax, mdone);
    tc_group_convert_kernel<<<dim3(nb, R_pad), 256, 0, st>>>(members, chunks, nchunks, V, R, R_pad, colmax,
                                                            static_cast<__half *>(V16), v_cols, vinv, mdone,
                                                            split ? 1 : 0);
    return check_launch("batched rhs conversion", 2);
}

// ===========================================================================
// Fused gradient estimator on tcgen05 (Eq. mll_grad with Eq. trace or
// Eq. pathwise_estimator):
//   g_l_k = (1/l_k) sum_ij phi_ij M_ij (a_ik - a_jk)^2,  g_sf = (2/s_f) sum_ij k_ij M_ij,
//   M_ij = sum_c lambda_c U_ci W_cj.
// Per 128-row x 64-column tile:
//   GEMM1  S = PA_I PB_J^T            (the kernel's exponent argument, as in the product)
//   GEMM-M M = U16_I W16_J^T          (K = right-hand sides, lambda folded into U16)
//   exp    W1 = phi' M (fp16, back into TMEM), row sums of W1, sum of k' M
//   GEMM3  D3 += W1 [A_J | A_J^2]     (hi/lo fp16 splits of the scaled coordinates)
// and per row i: sum_j W1_ij (a_ik - a_jk)^2 = a_ik^2 rs_i - 2 a_ik (W1 A)_ik + (W1 A^2)_ik,
// an exact identity for the rounded W1 (rs_i sums the same fp16 values).
// ===========================================================================
namespace {

constexpr int GTN = 64;  // gradient column tile

struct GParams {
    int KD, KM, N3p, d, nstages, nb3;
    int km_steps;  // K = 16 steps of GEMM-M that touch real right-hand sides (ceil(R / 16))
    int64_t n, col_tiles;
    int nsplit;
    // Symmetric sweep (sym_h > 0; U and W the same block, so M and the summand are symmetric
    // in i and j): only the column tiles from the row tile's diagonal block on, off-diagonal
    // tiles counted twice.  Row tile I's range [2I, 2 RT) is cut into ceil((RT - I) / sym_h)
    // near-equal items; CTA e takes item e (row tiles in order, so longer items come first).
    int64_t row_tiles, sym_h;
    const float *dscale;
    const float *guw;  // 1 / (G_u G_w)
    const float *X;
    float inv_ell[GP_MAX_D];
    float cphi_sf2;  // phi = cphi_sf2 * phi'  (3 s_f^2 Matern, s_f^2 RBF)
    float sf2;
    const float *inv_dev;  // device-resident 1/l and s_f^2 (replace inv_ell, sf2 when set)
    const float *sf2_dev;
    double *partial;
    int *err;
};

// F(M) = sum_{m=1..M} ceil(m / h): items of the row tiles with m = 1..M tiles pairs left.
__host__ __device__ __forceinline__ int64_t sym_items_upto(int64_t M, int64_t h) {
    const int64_t q = M / h, r = M - q * h;
    return h * q * (q + 1) / 2 + r * (q + 1);
}

// Item e of the symmetric sweep: row tile I (the largest with prefix(I) <= e, where
// prefix(I) = F(RT) - F(RT - I) items precede row tile I) and its column-tile range.
__device__ __forceinline__ void sym_item(int64_t e, int64_t RT, int64_t h, int64_t *I, int64_t *c0, int64_t *c1) {
    const int64_t FT = sym_items_upto(RT, h);
    int64_t lo = 0, hi = RT - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (FT - sym_items_upto(RT - mid, h) <= e) lo = mid;
        else hi = mid - 1;
    }
    const int64_t m = RT - lo, k = (m + h - 1) / h, part = e - (FT - sym_items_upto(m, h));
    const int64_t len = 2 * m;  // column tiles from 2 I to the end (64-column tiles, 128-row tiles)
    *I = lo;
    *c0 = 2 * lo + part * len / k;
    *c1 = 2 * lo + (part + 1) * len / k;
}

template <int KIND, int KAT>  // KAT: 64-wide atoms of the distance contraction (KD / 64)
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_grad_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapU, const __grid_constant__ CUtensorMap mapW,
                   const __grid_constant__ CUtensorMap mapB3, const GParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int katoms = p.KD / 64, matoms = p.KM / 64;
    const int NS = p.nstages;
    const uint32_t a_bytes = (uint32_t)TM * p.KD * 2, u_bytes = (uint32_t)TM * p.KM * 2;
    const uint32_t b_bytes = (uint32_t)GTN * p.KD * 2, w_bytes = (uint32_t)GTN * p.KM * 2;
    const uint32_t b3_bytes = (uint32_t)p.N3p * 128;
    const uint32_t stage_bytes = b_bytes + w_bytes;
    const int NB3 = p.nb3;
    // Two rings: PB/W tiles (read by GEMM1 and GEMM-M) and [A | A^2] tiles (read by GEMM3,
    // about two tiles later), each released by its own readers so neither holds the other.
    uint8_t *sA = smem;
    uint8_t *sU = sA + a_bytes;
    uint8_t *sStages = sU + u_bytes;
    uint8_t *sB3r = sStages + (size_t)NS * stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB3r + (size_t)NB3 * b3_bytes);
    uint64_t *a_full = bars;
    uint64_t *full = bars + 1;
    uint64_t *empty = full + MAX_STAGES;
    uint64_t *b3_full = empty + MAX_STAGES;
    uint64_t *b3_empty = b3_full + MAX_B3;
    // Three tile buffers in tensor memory, each holding S and M of a tile and then, written
    // over the S columns, the packed fp16 W1 of the same tile.
    uint64_t *t_full = b3_empty + MAX_B3;   // GEMM1 and GEMM-M of a tile landed (2 commits)
    uint64_t *t_kval = t_full + 3;          // the evaluation warpgroup wrote W1 into buffer b
    uint64_t *t_free = t_kval + 3;          // GEMM3 has consumed buffer b
    uint64_t *y_full = t_free + 3;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(y_full + 1);
    volatile int *s_err = reinterpret_cast<volatile int *>(tmem_slot + 1);
    double *red = reinterpret_cast<double *>(smem_raw);  // reused after the pipeline (reduction scratch)
    double *xch = reinterpret_cast<double *>(bars + 64);   // 256 doubles: per-row sums of warpgroup 1

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t row_tile, t0, t1;
    if (p.sym_h > 0) {
        sym_item(blockIdx.x, p.row_tiles, p.sym_h, &row_tile, &t0, &t1);
    } else {
        const int64_t per = cdiv(p.col_tiles, p.nsplit);
        row_tile = blockIdx.x;
        t0 = (int64_t)blockIdx.y * per;
        t1 = min(p.col_tiles, t0 + per);
    }
    const int64_t row0 = row_tile * TM;
    const int ntiles = (int)max((int64_t)0, t1 - t0);
    // symmetric sweep: column tiles past the diagonal block count twice (log2 weight 1)
    const int64_t twice_from = p.sym_h > 0 ? 2 * row_tile + 2 : INT64_MAX;

    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        for (int s = 0; s < MAX_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 2);  // released by the GEMM1 and GEMM-M issuers
        }
        for (int q = 0; q < MAX_B3; ++q) {
            mbar_init(&b3_full[q], 1);
            mbar_init(&b3_empty[q], 1);
        }
        for (int b = 0; b < 3; ++b) {
            mbar_init(&t_full[b], 2);
            mbar_init(&t_kval[b], 128);
            mbar_init(&t_free[b], 1);
        }
        mbar_init(y_full, 1);
        *s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // Tensor memory: tile buffers 0..2 at columns 0 / 128 / 256, each with S at +0 (W1
    // packed over its first 32 columns) and M at +64; the D3 accumulator at 384 (N3p <= 128).
    const uint32_t tmem = *tmem_slot;
    const uint32_t tS = tmem, tD = tmem + 384;

    double g_acc[1];  // silence unused warnings in non-epilogue warps
    (void)g_acc;
    float gk[64];
    double rs_acc = 0.0, s_acc = 0.0;

    // The role warps (0, 1, 2, 3, 12) run their loops with the whole warp (warp-uniform waits
    // and loop state) and issue TMA, MMA and commit instructions from one elected lane.
    if (warp == 0 && ntiles > 0) {
        const bool leader = elect_one();
        if (leader) {
            mbar_expect_tx(a_full, a_bytes + u_bytes);
            for (int ka = 0; ka < katoms; ++ka) tma_load_2d(sA + ka * (TM * 128), &mapA, a_full, ka * 64, (int)row0);
            for (int ka = 0; ka < matoms; ++ka) tma_load_2d(sU + ka * (TM * 128), &mapU, a_full, ka * 64, (int)row0);
        }
        __syncwarp();
        for (int it = 0; it < ntiles; ++it) {
            const int s = it % NS, use = it / NS;
            if (it >= NS && !mbar_wait_warp(&empty[s], (use - 1) & 1, s_err)) break;
            const int j0 = (int)((t0 + it) * GTN);
            uint8_t *sB = sStages + (size_t)s * stage_bytes;
            uint8_t *sW = sB + b_bytes;
            if (leader) {
                mbar_expect_tx(&full[s], stage_bytes);
                for (int ka = 0; ka < katoms; ++ka) tma_load_2d(sB + ka * (GTN * 128), &mapB, &full[s], ka * 64, j0);
                for (int ka = 0; ka < matoms; ++ka) tma_load_2d(sW + ka * (GTN * 128), &mapW, &full[s], ka * 64, j0);
            }
            __syncwarp();
        }
    } else if (warp == 12 && ntiles > 0) {
        // ------------------------------------------------ TMA producer: [A | A^2] ring
        const bool leader = elect_one();
        for (int it = 0; it < ntiles; ++it) {
            const int q = it % NB3;
            if (it >= NB3 && !mbar_wait_warp(&b3_empty[q], ((it / NB3) - 1) & 1, s_err)) break;
            const int j0 = (int)((t0 + it) * GTN);
            if (leader) {
                mbar_expect_tx(&b3_full[q], b3_bytes);
                tma_load_2d(sB3r + (size_t)q * b3_bytes, &mapB3, &b3_full[q], j0, 0);
            }
            __syncwarp();
        }
    } else if ((warp == 1 || warp == 2) && ntiles > 0) {
        // GEMM1 (warp 1) and GEMM-M (warp 2) issuers; GEMM3 has a third warp (3).
        // Three short issue streams instead of one long one; each stage and each tile buffer
        // is released by a commit of every warp that read it (empty[] and t_full[] count 2).
        const bool leader = elect_one();
        const uint32_t id1 = idesc_f16(TM, GTN);
        // descriptors built once, advanced in 16-byte units (single-thread issue paths)
        const uint64_t dA = sdesc(sA), dU = sdesc(sU), dSt = sdesc(sStages);
        const uint32_t st_units = stage_bytes >> 4, b_units = b_bytes >> 4;
        constexpr uint32_t a_atom = (TM * 128) >> 4, g_atom = (GTN * 128) >> 4;
        const bool is_g1 = (warp == 1);
        bool ok = mbar_wait_warp(a_full, 0, s_err);
        for (int it = 0; ok && it < ntiles; ++it) {
            const int s = it % NS, b = it % 3;
            if (!mbar_wait_warp(&full[s], (it / NS) & 1, s_err)) break;
            if (it >= 3 && !mbar_wait_warp(&t_free[b], ((it / 3) - 1) & 1, s_err)) break;
            tc_fence_after();
            const uint64_t dB = dSt + (uint64_t)s * st_units;
            if (!leader) {
            } else if (is_g1) {
#pragma unroll
                for (int k = 0; k < 4 * KAT; ++k) {
                    const uint32_t ka = (uint32_t)(k >> 2), ko = (uint32_t)(k & 3) * 2;
                    mma_ss(tS + b * 128, dA + ka * a_atom + ko, dB + ka * g_atom + ko, id1, k > 0 ? 1u : 0u);
                }
            } else {
                const uint64_t dW = dB + b_units;
                const int km = p.km_steps;  // the zero-padded columns beyond R are skipped
                for (int k = 0; k < km; ++k) {
                    const uint32_t ka = (uint32_t)(k >> 2), ko = (uint32_t)(k & 3) * 2;
                    mma_ss(tS + b * 128 + 64, dU + ka * a_atom + ko, dW + ka * g_atom + ko, id1, k > 0 ? 1u : 0u);
                }
            }
            if (leader) {
                mma_commit(&empty[s]);
                mma_commit(&t_full[b]);
            }
            __syncwarp();
        }
    } else if (warp == 3 && ntiles > 0) {
        // GEMM3 issuer: D3 += W1 [A | A^2]
        const bool leader = elect_one();
        const uint32_t id3 = idesc_f16(TM, p.N3p);
        const uint64_t dB3r = sdesc(sB3r);
        const uint32_t b3_units = b3_bytes >> 4;
        for (int it = 0; it < ntiles; ++it) {
            const int q = it % NB3, b = it % 3;
            if (!mbar_wait_warp(&b3_full[q], (it / NB3) & 1, s_err)) break;
            if (!mbar_wait_warp(&t_kval[b], (it / 3) & 1, s_err)) break;
            tc_fence_after();
            const uint64_t dB3 = dB3r + (uint64_t)q * b3_units;
            if (leader) {
#pragma unroll
                for (int k = 0; k < GTN / 16; ++k)
                    mma_ts(tD, tS + b * 128 + k * 8, dB3 + (uint32_t)k * 2, id3, (it > 0 || k > 0) ? 1u : 0u);
                mma_commit(&b3_empty[q]);
                mma_commit(&t_free[b]);
            }
            __syncwarp();
        }
        if (leader) mma_commit(y_full);
        __syncwarp();
    } else if (warp >= 4 && warp < 12) {
        // two evaluation warpgroups; warpgroup wg takes the tiles with it % 2 == wg (buffer
        // it % 3).  Each thread owns one row and writes the 32 packed W1 columns of a chunk
        // over S columns it has already read.
        const int wg = (warp - 4) >> 2;
        const int wq = warp & 3;
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        const float dsc = *p.dscale;
        bool ok = true;
        for (int it = wg; it < ntiles; it += 2) {
            const int b = it % 3;
            if (!mbar_wait(&t_full[b], (it / 3) & 1, s_err)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t taS = tS + b * 128 + lane_off, taM = taS + 64;
            const uint32_t taP = taS;
            const float cw = (t0 + it >= twice_from) ? 1.0f : 0.0f;  // log2 of the tile's weight
            float rs = 0.0f, sk = 0.0f;
#pragma unroll 1
            for (int ch = 0; ch < GTN / 32; ++ch) {
                uint32_t rS[32], rM[32];
                tmem_ld32(taS + ch * 32, rS);
                tmem_ld32(taM + ch * 32, rM);
                tmem_ld_wait();
                uint32_t pk[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    float w[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float S = __uint_as_float(rS[2 * e + h]);
                        const float M = __uint_as_float(rM[2 * e + h]);
                        float kp_, phi_;
                        if (KIND == GP_RBF) {
                            kp_ = ex2_approx(fminf(fmaf(S, dsc, cw), cw));
                            phi_ = kp_;
                        } else {
                            float u = fmaxf(S * dsc, 1e-30f);
                            float q = u * rsqrt_approx(u);
                            phi_ = ex2_approx(cw - q);
                            kp_ = fmaf(q, kLn2, 1.0f) * phi_;
                        }
                        w[h] = phi_ * M;
                        sk = fmaf(kp_, M, sk);
                    }
                    pk[e] = pack_half2(w[0], w[1]);
                    __half2 hw = *reinterpret_cast<__half2 *>(&pk[e]);
                    float2 fw = __half22float2(hw);
                    rs += fw.x + fw.y;
                }
                tmem_st16(taP + ch * 16, pk);
            }
            if (!ok) break;
            tmem_st_wait();
            tc_fence_before();
            mbar_arrive(&t_kval[b]);
            rs_acc += (double)rs;
            s_acc += (double)sk;
        }
        // combine the two warpgroups' per-row sums (named barrier over the 256 evaluation threads)
        const int row = wq * 32 + lane;
        if (wg == 1) {
            xch[row] = rs_acc;
            xch[128 + row] = s_acc;
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (wg == 0) {
            rs_acc += xch[row];
            s_acc += xch[128 + row];
        } else {
            s_acc = 0.0;
            ok = false;
        }
        if (wg == 0 && ok && ntiles > 0) ok = mbar_wait(y_full, 0, s_err);
        // per-row contributions sum_j W1_ij (a_ik - a_jk)^2
        const int64_t i = row0 + wq * 32 + lane;
        const int d = p.d;
        for (int k = 0; k < 64; ++k) gk[k] = 0.0f;
        if (ok && ntiles > 0) {
            tc_fence_after();
            float a[64];
            for (int k = 0; k < d; ++k)
                a[k] = (i < p.n) ? p.X[i * d + k] * (p.inv_dev ? p.inv_dev[k] : p.inv_ell[k]) : 0.0f;
            for (int k = 0; k < d; ++k) gk[k] = a[k] * a[k] * (float)rs_acc;
            for (int f0 = 0; f0 < p.N3p; f0 += 16) {
                uint32_t r[16];
                tmem_ld16(tD + lane_off + f0, r);
                tmem_ld_wait();
                for (int e = 0; e < 16; ++e) {
                    const int f = f0 + e;
                    if (f >= 4 * d) break;
                    const int part = f / d, k = f - part * d;
                    const float v = __uint_as_float(r[e]);
                    if (part < 2) gk[k] -= 2.0f * a[k] * v;
                    else gk[k] += v;
                }
            }
            if (i >= p.n) {
                for (int k = 0; k < d; ++k) gk[k] = 0.0f;
                s_acc = 0.0;
            }
        } else {
            s_acc = 0.0;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
    // block reduction over the 128 epilogue threads, fixed order
    double *out = p.partial + (int64_t)(blockIdx.y * gridDim.x + blockIdx.x) * (p.d + 1);
    const double sf2v = p.sf2_dev ? (double)*p.sf2_dev : (double)p.sf2;
    const double cphi = p.sf2_dev ? (KIND == GP_RBF ? 1.0 : 3.0) * sf2v : (double)p.cphi_sf2;
    const double gscale = cphi * (double)(*p.guw);
    const double sscale = sf2v * (double)(*p.guw);
    for (int k = 0; k <= p.d; ++k) {
        double v = 0.0;
        if (warp >= 4 && warp < 8) v = (k < p.d) ? (double)gk[k] * gscale : s_acc * sscale;
        v = warp_sum(v);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) out[k] = red[4] + red[5] + red[6] + red[7];
    }
    if (threadIdx.x == 0 && *s_err && p.err) atomicExch(p.err, 1);
}

// max |lambda_c U_ci| and max |W_cj| over i < n, c < R (float bits).
// grid (blocks over points, R): column c = blockIdx.y
__global__ void tc_uw_bound_kernel(GradArgs<float> a, unsigned int *bnd) {
    float mu = 0.0f, mw = 0.0f;
    const int64_t n = a.n;
    const int c = blockIdx.y;
    const float *uc = (c == 0) ? a.U0 : a.U + (int64_t)(c - 1) * a.ldu;
    const float *wc = (c == 0) ? a.W0 : a.W + (int64_t)(c - 1) * a.ldw;
    const float lam = (float)((c == 0) ? a.lam0 : a.lam_rest);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        mu = fmaxf(mu, fabsf(uc[i] * lam));
        mw = fmaxf(mw, fabsf(wc[i]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
    }
    // one atomic per block and bound (same-address atomics serialise)
    __shared__ float s_u[32], s_w[32];
    if ((threadIdx.x & 31) == 0) {
        s_u[threadIdx.x >> 5] = mu;
        s_w[threadIdx.x >> 5] = mw;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mu = fmaxf(mu, s_u[w]);
            mw = fmaxf(mw, s_w[w]);
        }
        atomicMax(&bnd[0], __float_as_uint(mu));
        atomicMax(&bnd[1], __float_as_uint(mw));
    }
}

__device__ __forceinline__ float pow2_norm(float m) {  // 2^-e with m 2^-e in [1, 2); 1 for 0 / non-finite
    if (!(m > 0.0f) || !isfinite(m)) return 1.0f;
    int e;
    frexpf(m, &e);
    return ldexpf(1.0f, 1 - e);
}

// U16[i][c] = fp16(lambda_c U_ci G_u), W16[j][c] = fp16(W_cj G_w), [n_pad x KM]; guw = 1/(G_u G_w).
// A block transposes 64 points x 64 columns at a time through shared memory: reads along the
// points of a column, writes along the columns of a point (both coalesced).  grid: point tiles.
__global__ void tc_uw_convert_kernel(GradArgs<float> a, int64_t n_pad, int KM, const unsigned int *bnd, __half *U16,
                                     __half *W16, float *guw) {
    __shared__ float tu[64][65], tw[64][65];
    const float gu = pow2_norm(__uint_as_float(bnd[0]));
    const float gw = pow2_norm(__uint_as_float(bnd[1]));
    if (blockIdx.x == 0 && threadIdx.x == 0) *guw = 1.0f / (gu * gw);
    const int64_t n = a.n;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 256 threads: 64 x 4
    for (int64_t i0 = (int64_t)blockIdx.x * 64; i0 < n_pad; i0 += (int64_t)gridDim.x * 64) {
        for (int c0 = 0; c0 < KM; c0 += 64) {
            __syncthreads();
            for (int cc = ty; cc < 64; cc += 4) {  // read: point i0 + tx of column c0 + cc
                const int c = c0 + cc;
                const int64_t i = i0 + tx;
                float u = 0.0f, w = 0.0f;
                if (i < n && c < a.R) {
                    u = (c == 0) ? a.U0[i] * (float)a.lam0 : a.U[(int64_t)(c - 1) * a.ldu + i] * (float)a.lam_rest;
                    w = (c == 0) ? a.W0[i] : a.W[(int64_t)(c - 1) * a.ldw + i];
                }
                tu[cc][tx] = u;
                tw[cc][tx] = w;
            }
            __syncthreads();
            for (int ii = ty; ii < 64; ii += 4) {  // write: column c0 + tx of point i0 + ii
                const int64_t e = (i0 + ii) * KM + c0 + tx;
                U16[e] = __float2half_rn(tu[tx][ii] * gu);
                W16[e] = __float2half_rn(tw[tx][ii] * gw);
            }
        }
    }
}

// B3[f][j] (N3p x n_pad): f = part * d + k, parts hi(a), lo(a), hi(a^2), lo(a^2) of a_jk = x_jk / l_k.
// grid (blocks over points, N3p): row f = blockIdx.y.
__global__ void tc_b3_kernel(const KP<float> kp, const float *X, int64_t n, int64_t n_pad, int N3p, __half *B3,
                             const float *inv_dev) {
    const int d = kp.d, f = blockIdx.y;
    const int part = f / d, k = f - part * d;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_pad; j += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.0f;
        if (j < n && f < 4 * d) {
            const float a = X[j * d + k] * (inv_dev ? inv_dev[k] : kp.inv_ell[k]);
            const float x = (part < 2) ? a : a * a;
            const __half h = __float2half_rn(x);
            v = (part & 1) ? (x - __half2float(h)) : __half2float(h);
        }
        B3[(int64_t)f * n_pad + j] = __float2half_rn(v);
    }
}

struct GradPlanTc {
    int KD, KM, N3p, ns, nb3, nsplit;
    int64_t n_pad, row_tiles, col_tiles;
    int64_t sym_h, sym_items;  // symmetric sweep: tile pairs per item (x 2 column tiles), items
    int64_t max_blocks;        // CTAs (partial sums) the workspace provides for
    size_t smem;
};
constexpr int kGradMaxSplit = 8;  // column splits per row tile the gradient's workspace covers

template <int KIND, int KAT>
int launch_grad_kernel(dim3 grid, size_t smem, const CUtensorMap &mA, const CUtensorMap &mB, const CUtensorMap &mU,
                       const CUtensorMap &mW, const CUtensorMap &mB3, const GParams &p, cudaStream_t st) {
    GP_TRY(ensure_max_dyn_smem((const void *)tc_grad_kernel<KIND, KAT>));
    tc_grad_kernel<KIND, KAT><<<grid, NTHREADS, smem, st>>>(mA, mB, mU, mW, mB3, p);
    return GP_OK;
}

GradPlanTc plan_tc_grad(int64_t n, int d, int R) {
    GradPlanTc g;
    g.KD = kd_for(d);
    g.KM = (int)rup(R, 64);
    g.N3p = (int)rup(4 * d, 16);
    g.n_pad = rup(std::max<int64_t>(n, 1), TM);
    g.row_tiles = g.n_pad / TM;
    g.col_tiles = g.n_pad / GTN;
    g.nsplit = pick_uniform_split(g.row_tiles, g.col_tiles, nullptr);
    // symmetric sweep: about six waves of items over the SMs, at least 8 tile pairs per item
    // (a CTA's fixed start-up and epilogue cost about four tiles)
    const int64_t waves = 6 * (int64_t)num_sms_tc();
    g.sym_h = std::max<int64_t>(8, cdiv(g.row_tiles * g.row_tiles, 2 * waves));
    g.sym_items = sym_items_upto(g.row_tiles, g.sym_h);
    // room for the autotuner's candidates: up to kGradMaxSplit splits, up to 32 waves of items
    g.max_blocks = std::max<int64_t>(g.row_tiles * std::max(g.nsplit, kGradMaxSplit),
                                     std::max<int64_t>(g.sym_items, 32 * (int64_t)num_sms_tc()));
    const size_t a = (size_t)TM * g.KD * 2 + (size_t)TM * g.KM * 2;
    const size_t st = (size_t)GTN * g.KD * 2 + (size_t)GTN * g.KM * 2;
    const size_t b3 = (size_t)g.N3p * 128;
    const size_t budget = kMaxDynSmem - 1024 - 512 - 2048 - a;  // alignment, barriers, row-sum exchange
    g.nb3 = (int)std::min<size_t>(6, std::max<size_t>(2, budget / 3 / b3));
    g.ns = (int)std::min<size_t>(MAX_STAGES, (budget - (size_t)g.nb3 * b3) / st);
    g.smem = 1024 + a + (size_t)g.ns * st + (size_t)g.nb3 * b3 + 512 + 2048;
    return g;
}

}  // namespace

// The tensor-core estimator covers d <= 32 (D3 accumulator of 4d columns next to three
// 128-column tile buffers in tensor memory) and s + 1 <= 256; wider problems use the
// CUDA-core FP32 reduction.
bool tc_grad_fits(int64_t n, int d, int R) {
    if (d > 32 || R > 256) return false;
    const GradPlanTc g = plan_tc_grad(n, d, R);
    return g.ns >= 2 && g.nb3 >= 2;
}

size_t tc_grad_workspace(int64_t n, int d, int R) {
    if (!tc_grad_fits(n, d, R)) return grad_simt_workspace<float>(n, d, R);
    GradPlanTc g = plan_tc_grad(n, d, R);
    Carver c(nullptr);
    c.take<char>(tc_points_bytes(n, d));
    c.take<__half>((size_t)g.n_pad * g.KM);
    c.take<__half>((size_t)g.n_pad * g.KM);
    c.take<__half>((size_t)g.N3p * g.n_pad);
    c.take<unsigned int>(2);
    c.take<float>(1);
    c.take<int>(1);
    c.take<double>((size_t)g.max_blocks * (d + 1));
    c.take<double>(256);
    return c.bytes();
}

int tc_grad(const GradArgs<float> &a, void *ws, size_t ws_bytes, cudaStream_t st) {
    const int d = a.kp.d;
    if (!tc_grad_fits(a.n, d, a.R)) return grad_simt<float>(a, ws, ws_bytes, st);
    GradPlanTc g = plan_tc_grad(a.n, d, a.R);
    if (g.ns < 2 || g.nb3 < 2) {
        set_error("tensor-core gradient tile does not fit shared memory");
        return GP_ERR_UNSUPPORTED;
    }
    Carver c(ws);
    void *pbuf = c.take<char>(tc_points_bytes(a.n, d));
    __half *U16 = c.take<__half>((size_t)g.n_pad * g.KM);
    __half *W16 = c.take<__half>((size_t)g.n_pad * g.KM);
    __half *B3 = c.take<__half>((size_t)g.N3p * g.n_pad);
    unsigned int *bnd = c.take<unsigned int>(2);
    float *guw = c.take<float>(1);
    c.take<int>(1);  // (kept for the workspace layout)
    int *err = tc_timeout_word();
    // U and W the same block with one lambda per column (the pathwise estimator): M and the
    // summand are symmetric in i and j, so the upper triangle of tiles suffices
    const bool sym = a.U0 == a.W0 && a.U == a.W && (a.R == 1 || a.ldu == a.ldw);
    // work split: forced (autotuner), tuned, or the built-in rule -- within the workspace
    {
        int64_t v = g_force_grad != 0 ? g_force_grad : tune_get(TuneKey{1, g.KD, g.KM, g.row_tiles, sym ? 1 : 0});
        if (sym && v >= 1 && sym_items_upto(g.row_tiles, v) <= g.max_blocks) {
            g.sym_h = v;
            g.sym_items = sym_items_upto(g.row_tiles, v);
        } else if (!sym && v >= 1 && v <= g.col_tiles && g.row_tiles * v <= g.max_blocks) {
            g.nsplit = (int)v;
        }
    }
    const int nblocks = (int)(sym ? g.sym_items : g.row_tiles * g.nsplit);
    double *partial = c.take<double>((size_t)g.max_blocks * (d + 1));
    double *dpart = c.take<double>(256);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));

    TcPoints pts;
    GP_TRY(tc_prepare_points_dev(a.kp, a.X, a.n, pbuf, &pts, a.dev_inv_ell, st));
    GP_TRY_CUDA(cudaMemsetAsync(bnd, 0, 2 * sizeof(unsigned int), st));
    tc_uw_bound_kernel<<<dim3((unsigned)std::min<int64_t>(cdiv(a.n, 1024), 256), (unsigned)a.R), 256, 0, st>>>(a, bnd);
    tc_uw_convert_kernel<<<(unsigned)std::min<int64_t>(cdiv(g.n_pad, 64), 1024), 256, 0, st>>>(a, g.n_pad, g.KM, bnd,
                                                                                             U16, W16, guw);
    tc_b3_kernel<<<dim3((unsigned)std::min<int64_t>(cdiv(g.n_pad, 1024), 256), (unsigned)g.N3p), 256, 0, st>>>(
        a.kp, a.X, a.n, g.n_pad, g.N3p, B3, a.dev_inv_ell);
    GP_TRY(check_launch("tc gradient operand preparation", 3));

    CUtensorMap mA, mB, mU, mW, mB3;
    GP_TRY(make_map(&mA, pts.PA, g.KD, g.n_pad, 64, TM));
    GP_TRY(make_map(&mB, pts.PB, g.KD, g.n_pad, 64, GTN));
    GP_TRY(make_map(&mU, U16, g.KM, g.n_pad, 64, TM));
    GP_TRY(make_map(&mW, W16, g.KM, g.n_pad, 64, GTN));
    GP_TRY(make_map(&mB3, B3, g.n_pad, g.N3p, 64, g.N3p));
    GParams p{};
    p.KD = g.KD;
    p.KM = g.KM;
    p.km_steps = (int)cdiv(a.R, 16);
    p.N3p = g.N3p;
    p.d = d;
    p.nstages = g.ns;
    p.nb3 = g.nb3;
    p.n = a.n;
    p.col_tiles = g.col_tiles;
    p.nsplit = g.nsplit;
    p.dscale = pts.dscale;
    p.guw = guw;
    p.X = a.X;
    for (int k = 0; k < d; ++k) p.inv_ell[k] = a.kp.inv_ell[k];
    p.cphi_sf2 = (a.kp.kind == GP_RBF ? 1.0f : 3.0f) * a.kp.sf2;
    p.inv_dev = a.dev_inv_ell;
    p.sf2_dev = a.dev_sf2;
    p.sf2 = a.kp.sf2;
    p.partial = partial;
    p.err = err;
    p.row_tiles = g.row_tiles;
    p.sym_h = sym ? g.sym_h : 0;
    dim3 grid = sym ? dim3((unsigned)g.sym_items, 1) : dim3((unsigned)g.row_tiles, (unsigned)g.nsplit);
    const int kat = g.KD / 64;  // <= 2 since d <= 32
    prof_begin(st, 1);
    if (a.kp.kind == GP_RBF) {
        if (kat == 1) GP_TRY(launch_grad_kernel<GP_RBF, 1>(grid, g.smem, mA, mB, mU, mW, mB3, p, st));
        else if (kat == 2) GP_TRY(launch_grad_kernel<GP_RBF, 2>(grid, g.smem, mA, mB, mU, mW, mB3, p, st));
        else GP_TRY(launch_grad_kernel<GP_RBF, 3>(grid, g.smem, mA, mB, mU, mW, mB3, p, st));
    } else {
        if (kat == 1) GP_TRY(launch_grad_kernel<GP_MATERN32, 1>(grid, g.smem, mA, mB, mU, mW, mB3, p, st));
        else if (kat == 2) GP_TRY(launch_grad_kernel<GP_MATERN32, 2>(grid, g.smem, mA, mB, mU, mW, mB3, p, st));
        else GP_TRY(launch_grad_kernel<GP_MATERN32, 3>(grid, g.smem, mA, mB, mU, mW, mB3, p, st));
    }
    prof_end(st);
    GP_TRY(check_launch("tc_grad_kernel"));
    return grad_tail<float>(a, nblocks, partial, dpart, st);
}

// Times the tensor-core gradient for a ladder of work splits (tile pairs per item of the
// symmetric sweep, or column splits per row tile) and records the fastest for the shape.
// Synchronises `st`; not for use inside a stream capture.
int tc_autotune_grad(const GradArgs<float> &a, int reps, void *ws, size_t ws_bytes, cudaStream_t st, int64_t *best_v,
                     double *best_ms) {
    const int d = a.kp.d;
    if (!tc_grad_fits(a.n, d, a.R)) {
        set_error("autotune: the tensor-core gradient does not cover d=%d, R=%d", d, a.R);
        return GP_ERR_UNSUPPORTED;
    }
    const GradPlanTc g = plan_tc_grad(a.n, d, a.R);
    const bool sym = a.U0 == a.W0 && a.U == a.W && (a.R == 1 || a.ldu == a.ldw);
    std::vector<int64_t> cand;
    if (sym) {
        const int64_t RT = g.row_tiles, sms = num_sms_tc();
        for (double w : {1.0, 1.5, 2.0, 3.0, 4.0, 6.0, 8.0, 12.0, 16.0, 24.0, 32.0}) {
            const int64_t h = std::max<int64_t>(2, (int64_t)std::ceil((double)RT * RT / (2.0 * w * sms)));
            if (sym_items_upto(RT, h) <= g.max_blocks) cand.push_back(h);
        }
    } else {
        for (int k = 1; k <= kGradMaxSplit; ++k)
            if (k <= g.col_tiles && g.row_tiles * k <= g.max_blocks) cand.push_back(k);
    }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GP_TRY_CUDA(cudaEventCreate(&e0));
    GP_TRY_CUDA(cudaEventCreate(&e1));
    int64_t best = 0;
    double best_t = 1e300;
    int rc = GP_OK;
    for (int64_t v : cand) {
        g_force_grad = v;
        double t_min = 1e300;
        for (int r = 0; r <= reps && rc == GP_OK; ++r) {  // the first run is a warm-up
            if (cudaEventRecord(e0, st) != cudaSuccess) rc = GP_ERR_CUDA;
            if (rc == GP_OK) rc = tc_grad(a, ws, ws_bytes, st);
            if (rc == GP_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = GP_ERR_CUDA;
            if (rc == GP_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = GP_ERR_CUDA;
            float ms = 0.0f;
            if (rc == GP_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = GP_ERR_CUDA;
            if (rc == GP_OK && r > 0) t_min = std::min(t_min, (double)ms);
        }
        g_force_grad = 0;
        if (rc != GP_OK) break;
        if (t_min < best_t) {
            best_t = t_min;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GP_OK) {
        set_error("autotune: a timed gradient failed");
        return rc;
    }
    if (best == 0) {
        set_error("autotune: no candidate work split");
        return GP_ERR_UNSUPPORTED;
    }
    GP_TRY(tune_put(TuneKey{1, g.KD, g.KM, g.row_tiles, sym ? 1 : 0}, best));
    *best_v = best;
    *best_ms = best_t;
    return GP_OK;
}

}  // namespace gp
