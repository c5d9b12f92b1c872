// Random Fourier features on the tensor cores (App. B "Kernel Function and Random Features").
#include "gp_internal.cuh"
#include "tcgen05.cuh"

#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>

namespace gp {

// ===========================================================================
// Random Fourier features on the tensor cores (App. B "Kernel Function and Random
// Features").  F^T = Phi W'^T over K = m features: Phi[i][2l] = cos(w_l . x_i) and
// Phi[i][2l+1] = sin(w_l . x_i) (the pair of frequency l side by side, W' permuted to
// match).  Both operands are split into fp16 hi + lo parts and the product is taken as
// hi.hi + hi.lo + lo.hi with FP32 accumulation in tensor memory (the dropped lo.lo term is
// ~2^-22 relative), which keeps FP32-level accuracy at the fp16 tensor rate.  Per CTA: 128
// points; 256 threads compute the features of 32 frequencies (one 64-feature, 128-byte
// swizzle atom) per K-chunk straight into shared memory, warp 0 streams the weight tiles
// by TMA, one thread of warp 1 issues the MMAs; every wait is bounded.
// ===========================================================================
namespace {

constexpr int RF_THREADS = 384;
constexpr int RF_NA = 3;     // feature-tile stages
constexpr int RF_FREQ = 32;  // frequencies per K-chunk
constexpr int RF_MAXD = 32;  // point coordinates held in registers
constexpr int RF_MAXS = 128; // samples (accumulator columns)

struct RfParams {
    int64_t n;
    int d, nchunks, s, s_pad, nb;
    uint32_t tcols;
    const float *X;   // n x d
    const float *Om;  // (nchunks * RF_FREQ) x d scaled frequencies (zero rows past m/2)
    float amp;        // s_f sqrt(2 / m)
    float *F;
    int64_t ldf;
    int *err;
};

// sin and cos of a: Cody-Waite reduction by 2 pi with a two-term split of 2 pi (Cody & Waite,
// "Software Manual for the Elementary Functions", 1980) to r in [-pi, pi], then the MUFU
// approximations, whose absolute error on that interval is below 2^-20.
__device__ __forceinline__ void rf_sincos(float a, float *sn, float *cs) {
    const float q = rintf(a * 0.15915494309189535f);
    float r = fmaf(-q, 6.28318548202514648f, a);  // 2 pi rounded to float ...
    r = fmaf(-q, -1.7484556000744883e-7f, r);      // ... and the rest of 2 pi
    asm("sin.approx.f32 %0, %1;" : "=f"(*sn) : "f"(r));
    asm("cos.approx.f32 %0, %1;" : "=f"(*cs) : "f"(r));
}

__device__ __forceinline__ void rf_split(float v, __half *hi, __half *lo) {
    const __half h = __float2half_rn(v);
    *hi = h;
    *lo = __float2half_rn(v - __half2float(h));
}

// Om[l][k] = omega_hat[l][k] / l_k (* sqrt(3 / chi2_l) for Matern-3/2), rows of dp = 4 ceil(d/4)
// floats (zero past d and past m/2);
// Wt[r][k], r < s_pad: hi part of w(r, k); r >= s_pad: lo part of w(r - s_pad, k), with
// w(j, 2l + e) = W[j][e m/2 + l] (zero for j >= s or l >= m/2).
__global__ void tc_rff_prep_kernel(const KP<float> kp, int m, const float *omega_hat, const float *chi2,
                                   const float *W, int s, int s_pad, int h_pad, int dp, float *Om, __half *Wt) {
    const int d = kp.d, h = m / 2;
    const int64_t nom = (int64_t)h_pad * dp, mp = 2 * (int64_t)h_pad, nw = (int64_t)s_pad * mp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nom + nw;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nom) {
            const int l = (int)(e / dp), k = (int)(e - (int64_t)l * dp);
            float w = 0.0f;
            if (l < h && k < d) {
                const float t = (kp.kind == GP_MATERN32) ? sqrtf(3.0f / chi2[l]) : 1.0f;
                w = omega_hat[(int64_t)l * d + k] * kp.inv_ell[k] * t;
            }
            Om[e] = w;
        } else {
            const int64_t q = e - nom;
            const int j = (int)(q / mp), kk = (int)(q - (int64_t)j * mp);
            const int l = kk >> 1, odd = kk & 1;
            const float v = (j < s && l < h) ? W[(int64_t)j * m + (int64_t)odd * h + l] : 0.0f;
            __half hi, lo;
            rf_split(v, &hi, &lo);
            Wt[(int64_t)j * mp + kk] = hi;
            Wt[(int64_t)(s_pad + j) * mp + kk] = lo;
        }
    }
}


// DQ: float4 groups per frequency row (d <= 4 DQ; 1, 2, 4 or 8), fixed so that the dot
// products are fully unrolled without predicated-off steps.
template <int DQ>
__global__ void __launch_bounds__(RF_THREADS, 1) tc_rff_kernel(const __grid_constant__ CUtensorMap mapW,
                                                                const RfParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr uint32_t a_bytes = 128 * 128;  // one fp16 feature tile: 128 points x 64 features
    const uint32_t w_bytes = (uint32_t)p.s_pad * 128;
    uint8_t *sA = smem;                              // RF_NA stages x {hi, lo}
    uint8_t *sW = sA + RF_NA * 2 * a_bytes;          // nb stages x {hi, lo}
    // each weight stage also carries its chunk's frequencies (RF_FREQ rows of 4 DQ floats)
    constexpr int dpd = 4 * DQ;
    const uint32_t om_bytes = (uint32_t)RF_FREQ * dpd * 4;
    float *sOm = reinterpret_cast<float *>(sW + (size_t)p.nb * 2 * w_bytes);
    uint64_t *a_full = reinterpret_cast<uint64_t *>(sOm + (size_t)p.nb * RF_FREQ * RF_MAXD);
    uint64_t *a_empty = a_full + RF_NA;
    uint64_t *w_full = a_empty + RF_NA;
    uint64_t *w_empty = w_full + 4;
    uint64_t *d_full = w_empty + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(d_full + 1);
    volatile int *s_err = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nch = p.nchunks;
    const int64_t row0 = (int64_t)blockIdx.x * 128;

    if (threadIdx.x == 0) {
        for (int k = 0; k < RF_NA; ++k) {
            mbar_init(&a_full[k], 8);
            mbar_init(&a_empty[k], 1);
        }
        for (int k = 0; k < 4; ++k) {
            mbar_init(&w_full[k], 1);
            mbar_init(&w_empty[k], 1);
        }
        mbar_init(d_full, 1);
        *s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(p.tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tD = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer: weight tiles (hi, lo)
        const bool leader = elect_one();
        for (int c = 0; c < nch; ++c) {
            const int s = c % p.nb;
            if (c >= p.nb && !mbar_wait_warp(&w_empty[s], ((c / p.nb) - 1) & 1, s_err)) break;
            if (leader) {
                uint8_t *dst = sW + (size_t)s * 2 * w_bytes;
                mbar_expect_tx(&w_full[s], 2 * w_bytes + om_bytes);
                tma_load_2d(dst, &mapW, &w_full[s], c * 64, 0);
                tma_load_2d(dst + w_bytes, &mapW, &w_full[s], c * 64, p.s_pad);
                bulk_load(sOm + (size_t)s * RF_FREQ * RF_MAXD, p.Om + (int64_t)c * RF_FREQ * dpd, om_bytes, &w_full[s]);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer: D += Phi_hi W_hi + Phi_hi W_lo + Phi_lo W_hi
        const bool leader = elect_one();
        const uint32_t id = idesc_f16(128, p.s_pad);
        const uint64_t dA = sdesc(sA), dW = sdesc(sW);
        for (int c = 0; c < nch; ++c) {
            const int sa = c % RF_NA, sw = c % p.nb;
            if (!mbar_wait_warp(&w_full[sw], (c / p.nb) & 1, s_err)) break;
            if (!mbar_wait_warp(&a_full[sa], (c / RF_NA) & 1, s_err)) break;
            tc_fence_after();
            if (leader) {
                const uint64_t ah = dA + ((uint64_t)sa * 2 * a_bytes >> 4), al = ah + (a_bytes >> 4);
                const uint64_t wh = dW + ((uint64_t)sw * 2 * w_bytes >> 4), wl = wh + (w_bytes >> 4);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t ko = (uint32_t)k * 2;
                    mma_ss(tD, ah + ko, wh + ko, id, (c > 0 || k > 0) ? 1u : 0u);
                    mma_ss(tD, ah + ko, wl + ko, id, 1u);
                    mma_ss(tD, al + ko, wh + ko, id, 1u);
                }
                mma_commit(&a_empty[sa]);
                mma_commit(&w_empty[sw]);
                if (c == nch - 1) mma_commit(d_full);
            }
            __syncwarp();
        }
    } else if (warp >= 4) {
        // ------------------------------------------------ features (256 threads) + epilogue
        // Thread (row, half): point row0 + row, frequencies 16 half .. 16 half + 15 of each
        // chunk, i.e. the 16-byte units 4 half .. 4 half + 3 of the row's 128-byte feature row,
        // stored at unit u ^ (row & 7) (the 128-byte swizzle the descriptors describe).
        const int ft = threadIdx.x - 128;
        const int row = ft & 127, half = ft >> 7;
        const int64_t ip = row0 + row;
        const int d = p.d;
        float x[4 * DQ];
#pragma unroll
        for (int k = 0; k < 4 * DQ; ++k) x[k] = (k < d && ip < p.n) ? p.X[ip * d + k] : 0.0f;
        bool ok = true;
        for (int c = 0; c < nch; ++c) {
            // the chunk's frequencies arrive with its weight tiles; the stage stays until the
            // MMAs of the chunk, which follow this chunk's features, have completed
            const int sw = c % p.nb, sa = c % RF_NA;
            if (!mbar_wait_warp(&w_full[sw], (c / p.nb) & 1, s_err)) {
                ok = false;
                break;
            }
            if (c >= RF_NA && !mbar_wait_warp(&a_empty[sa], ((c / RF_NA) - 1) & 1, s_err)) {
                ok = false;
                break;
            }
            const float *om_s = sOm + (size_t)sw * RF_FREQ * RF_MAXD;
            uint8_t *th = sA + (size_t)sa * 2 * a_bytes, *tl = th + a_bytes;
            const float4 *om4 = reinterpret_cast<const float4 *>(om_s + half * 16 * dpd);
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                // four frequencies at a time: independent dot products, then sin / cos
                float arg[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int k4 = 0; k4 < DQ; ++k4) {
#pragma unroll
                    for (int f4 = 0; f4 < 4; ++f4) {
                        const float4 w = om4[(q * 4 + f4) * DQ + k4];
                        arg[f4] = fmaf(w.x, x[4 * k4], arg[f4]);
                        arg[f4] = fmaf(w.y, x[4 * k4 + 1], arg[f4]);
                        arg[f4] = fmaf(w.z, x[4 * k4 + 2], arg[f4]);
                        arg[f4] = fmaf(w.w, x[4 * k4 + 3], arg[f4]);
                    }
                }
                uint32_t hv[4], lv[4];
#pragma unroll
                for (int f4 = 0; f4 < 4; ++f4) {
                    float sn, cs;
                    rf_sincos(arg[f4], &sn, &cs);
                    __half ch, cl, sh, sl;
                    rf_split(cs, &ch, &cl);
                    rf_split(sn, &sh, &sl);
                    __half2 h2 = __halves2half2(ch, sh), l2 = __halves2half2(cl, sl);
                    hv[f4] = *reinterpret_cast<uint32_t *>(&h2);
                    lv[f4] = *reinterpret_cast<uint32_t *>(&l2);
                }
                const uint32_t off = (uint32_t)row * 128 + ((uint32_t)((half * 4 + q) ^ (row & 7)) << 4);
                *reinterpret_cast<uint4 *>(th + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                *reinterpret_cast<uint4 *>(tl + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
            }
            // generic-proxy writes become visible to the tensor cores' async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_full[sa]);
        }
        if (ok) ok = mbar_wait(d_full, 0, s_err);
        if (ok) {
            tc_fence_after();
            const int wq = warp & 3, g = (warp - 4) >> 2;
            const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
            const int64_t i = row0 + wq * 32 + lane;
            for (int c0 = 16 * g; c0 < p.s_pad; c0 += 32) {
                uint32_t r[16];
                tmem_ld16(tD + lane_off + c0, r);
                tmem_ld_wait();
                if (i < p.n) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int j = c0 + e;
                        if (j < p.s) p.F[(int64_t)j * p.ldf + i] = p.amp * __uint_as_float(r[e]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tD), "r"(p.tcols) : "memory");
    }
    if (threadIdx.x == 0 && *s_err && p.err) atomicExch(p.err, 1);
}

// float4 groups per frequency row of the instantiation that serves d
int rf_dq(int d) { return d <= 4 ? 1 : d <= 8 ? 2 : d <= 16 ? 4 : 8; }

template <int DQ>
int launch_rff_kernel(const CUtensorMap &mW, const RfParams &p, size_t smem, int64_t grid, cudaStream_t st) {
    GP_TRY(ensure_max_dyn_smem((const void *)tc_rff_kernel<DQ>));
    tc_rff_kernel<DQ><<<(unsigned)grid, RF_THREADS, smem, st>>>(mW, p);
    return GP_OK;
}

struct RfPlan {
    int s_pad, h_pad, nb;
    uint32_t tcols;
    size_t smem;
};

RfPlan plan_rff(int m, int s) {
    RfPlan g{};
    g.s_pad = (int)rup(std::max(s, 1), 16);
    g.h_pad = (int)rup(m / 2, RF_FREQ);
    g.tcols = 32;
    while ((int)g.tcols < g.s_pad) g.tcols <<= 1;
    const size_t a = (size_t)RF_NA * 2 * 128 * 128, w = (size_t)2 * g.s_pad * 128;
    const size_t om = (size_t)RF_FREQ * RF_MAXD * 4;  // frequencies of one stage
    const size_t budget = kMaxDynSmem - 1024 - 256 - a;
    g.nb = (int)std::min<size_t>(4, budget / (w + om));
    g.smem = 1024 + a + (size_t)g.nb * (w + om) + 256;
    return g;
}

}  // namespace

bool tc_rff_fits(int d, int m, int s) {
    if (d > RF_MAXD || s > RF_MAXS || m < 2) return false;
    return plan_rff(m, s).nb >= 2;
}

size_t tc_rff_workspace(int d, int m, int s) {
    const RfPlan g = plan_rff(m, s);
    Carver c(nullptr);
    c.take<float>((size_t)g.h_pad * 4 * rf_dq(d));
    c.take<__half>((size_t)2 * g.s_pad * 2 * g.h_pad);
    c.take<int>(1);
    return c.bytes();
}

int tc_rff(const KP<float> &kp, const float *X, int64_t n, int m, const float *omega_hat, const float *chi2,
           const float *W, int s, float *F, int64_t ldf, void *ws, size_t ws_bytes, cudaStream_t st) {
    const int d = kp.d;
    const RfPlan g = plan_rff(m, s);
    Carver c(ws);
    float *Om = c.take<float>((size_t)g.h_pad * 4 * rf_dq(d));
    __half *Wt = c.take<__half>((size_t)2 * g.s_pad * 2 * g.h_pad);
    c.take<int>(1);  // (kept for the workspace layout)
    int *err = tc_timeout_word();
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    const int dp = 4 * rf_dq(d);
    const int64_t prep = (int64_t)g.h_pad * dp + (int64_t)g.s_pad * 2 * g.h_pad;
    tc_rff_prep_kernel<<<(unsigned)std::min<int64_t>(cdiv(prep, 256), 2048), 256, 0, st>>>(
        kp, m, omega_hat, chi2, W, s, g.s_pad, g.h_pad, dp, Om, Wt);
    GP_TRY(check_launch("tc_rff_prep_kernel"));
    CUtensorMap mW;
    GP_TRY(tc_make_map16(&mW, Wt, (uint64_t)2 * g.h_pad, (uint64_t)2 * g.s_pad, 64, (uint32_t)g.s_pad));
    RfParams p{};
    p.n = n;
    p.d = d;
    p.nchunks = g.h_pad / RF_FREQ;
    p.s = s;
    p.s_pad = g.s_pad;
    p.nb = g.nb;
    p.tcols = g.tcols;
    p.X = X;
    p.Om = Om;
    p.amp = kp.sf * sqrtf(2.0f / (float)m);
    p.F = F;
    p.ldf = ldf;
    p.err = err;
    const int dq = rf_dq(d);
    if (dq == 1) GP_TRY(launch_rff_kernel<1>(mW, p, g.smem, cdiv(n, 128), st));
    else if (dq == 2) GP_TRY(launch_rff_kernel<2>(mW, p, g.smem, cdiv(n, 128), st));
    else if (dq == 4) GP_TRY(launch_rff_kernel<4>(mW, p, g.smem, cdiv(n, 128), st));
    else GP_TRY(launch_rff_kernel<8>(mW, p, g.smem, cdiv(n, 128), st));
    return check_launch("tc_rff_kernel");
}

}  // namespace gp
