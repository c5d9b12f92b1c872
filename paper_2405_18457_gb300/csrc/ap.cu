// Alternating projections, Alg. 2 (App. B "Alternating Projections").
//
// Set-up per call (= per marginal-likelihood step): every diagonal block
// H[i, i] (block_size x block_size, the ragged last block padded with the
// identity) is materialised, Cholesky-factored and turned into its explicit
// inverse H[i,i]^-1 = L^-T L^-1 by blocked batched kernels (32-wide panels,
// the O(b^3) parts on a tiled batched GEMM).  The paper caches the Cholesky
// factor and applies chol_solve; the explicit inverse gives the same
// H[i,i]^-1 r[i] through one small matrix product per iteration instead of two
// sequential triangular solves.
//
// Iteration: block score ||sum_c r_c[i]|| -> argmax on the device -> delta =
// H[i,i]^-1 r[i] -> v[i] += delta -> r -= H[:, i] delta (kernel panel product
// with a device-resident column offset) -> split norms and loop condition.
#include "solver_common.cuh"

#include <algorithm>
#include <type_traits>

namespace gp {

namespace {

constexpr int PW = 32;  // panel width of the blocked factorisation

// ---------------------------------------------------------------- batched GEMM
// C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b], row-major, 64x64 tiles.  Structure of the
// factorisation's products (GemmShape): lower -- only output tiles on or below the diagonal
// (n0 <= m0) are computed; mirror -- each off-diagonal tile is also written transposed (a
// symmetric result); kfrom -- the K loop starts at n0 (op(B) lower-triangular: B[k][j] = 0 for
// k < j) or at max(m0, n0) (op(A) upper- and op(B) lower-triangular, as in Z^T Z for a lower-
// triangular Z).  Skipped terms are exact zeros, so the results equal the full products'.
struct GemmShape {
    int lower, mirror, kfrom;  // kfrom: 0 = from 0, 1 = from n0, 2 = from max(m0, n0)
};
template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_batched_kernel(int M, int N, int K, T alpha, const T *A, int lda,
                                                           int64_t sA, const T *B, int ldb, int64_t sB, T beta,
                                                           T *C, int ldc, int64_t sC, GemmShape shp) {
    __shared__ T As[16][64 + 1];
    __shared__ T Bs[16][64 + 1];
    const int b = blockIdx.z;
    A += b * sA;
    B += b * sB;
    C += b * sC;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    if (shp.lower && n0 > m0) return;
    const int kbeg = shp.kfrom == 0 ? 0 : (shp.kfrom == 1 ? n0 : max(m0, n0));
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k0 = kbeg; k0 < K; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            int kk = e / 64, mm = e % 64;
            int gm = m0 + mm, gk = k0 + kk;
            T v = T(0);
            if (gm < M && gk < K) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
            As[kk][mm] = v;
            int gn = n0 + mm;
            T w = T(0);
            if (gn < N && gk < K) w = TB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
            Bs[kk][mm] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            T *cp = C + (int64_t)gm * ldc + gn;
            const T y = alpha * acc[i][j] + (beta == T(0) ? T(0) : beta * *cp);
            *cp = y;
            if (shp.mirror && n0 < m0) C[(int64_t)gn * ldc + gm] = y;
        }
    }
}

template <typename T, bool TA, bool TB>
int gemm_batched(int M, int N, int K, T alpha, const T *A, int lda, int64_t sA, const T *B, int ldb, int64_t sB,
                 T beta, T *C, int ldc, int64_t sC, int batch, cudaStream_t st, GemmShape shp = GemmShape{0, 0, 0}) {
    if (M <= 0 || N <= 0) return GP_OK;
    dim3 grid((unsigned)cdiv(N, 64), (unsigned)cdiv(M, 64), (unsigned)batch);
    gemm_batched_kernel<T, TA, TB><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC,
                                                         shp);
    return check_launch("gemm_batched_kernel");
}

// H[b] block matrix: k(x_{lo+a}, x_{lo+a'}) + sigma^2 delta; padded rows -> identity.
template <typename T>
__global__ void ap_build_blocks_kernel(const KP<T> kp, const T *X, int64_t n, int bs, int bsp, T *Hb) {
    const int b = blockIdx.z;
    const int a = blockIdx.y * 16 + threadIdx.y;
    const int ap = blockIdx.x * 16 + threadIdx.x;
    if (a >= bsp || ap >= bsp) return;
    const int64_t lo = (int64_t)b * bs;
    const int64_t i = lo + a, j = lo + ap;
    T v;
    if (a >= bs || ap >= bs || i >= n || j >= n) {
        v = (a == ap) ? T(1) : T(0);
    } else {
        T r2 = T(0);
        for (int k = 0; k < kp.d; ++k) {
            T t = (X[i * kp.d + k] - X[j * kp.d + k]) * kp.inv_ell[k];
            r2 += t * t;
        }
        v = kval(kp.kind, kp.sf2, r2) + (a == ap ? kp.sigma2 : T(0));
    }
    Hb[(int64_t)b * bsp * bsp + (int64_t)a * bsp + ap] = v;
}

// Unblocked Cholesky of the 32x32 diagonal tile at (p, p), one warp per matrix.
template <typename T>
__global__ void potf2_kernel(T *Hb, int bsp, int p, int *fail) {
    __shared__ T L[PW][PW + 1];
    T *A = Hb + (int64_t)blockIdx.x * bsp * bsp;
    const int lane = threadIdx.x;
    for (int k = 0; k < PW; ++k) L[lane][k] = A[(int64_t)(p + lane) * bsp + p + k];
    __syncwarp();
    for (int j = 0; j < PW; ++j) {
        T djj = L[j][j];
        if (!(djj > T(0))) {
            if (lane == 0) atomicExch(fail, 1);
            djj = T(1);
        }
        T ljj = sqrt(djj);
        __syncwarp();
        if (lane == j) L[j][j] = ljj;
        if (lane > j) L[lane][j] = L[lane][j] / ljj;
        __syncwarp();
        if (lane > j)
            for (int k = j + 1; k <= lane; ++k) L[lane][k] -= L[lane][j] * L[k][j];
        __syncwarp();
    }
    for (int k = 0; k < PW; ++k) A[(int64_t)(p + lane) * bsp + p + k] = (k <= lane) ? L[lane][k] : T(0);
}

// Rows i >= p+32: A[i, p:p+32] <- A[i, p:p+32] L_pp^-T  (one thread per row).
template <typename T>
__global__ void trsm_right_kernel(T *Hb, int bsp, int p) {
    __shared__ T L[PW][PW + 1];
    T *A = Hb + (int64_t)blockIdx.x * bsp * bsp;
    for (int e = threadIdx.x; e < PW * PW; e += blockDim.x) L[e / PW][e % PW] = A[(int64_t)(p + e / PW) * bsp + p + e % PW];
    __syncthreads();
    const int i = p + PW + blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= bsp) return;
    T x[PW];
#pragma unroll
    for (int j = 0; j < PW; ++j) x[j] = A[(int64_t)i * bsp + p + j];
#pragma unroll
    for (int j = 0; j < PW; ++j) {
        T s = x[j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= x[k] * L[j][k];
        x[j] = s / L[j][j];
    }
#pragma unroll
    for (int j = 0; j < PW; ++j) A[(int64_t)i * bsp + p + j] = x[j];
}

// Z[p:p+32, 0:p+32] <- L_pp^-1 Z[p:p+32, 0:p+32]  (one thread per column).
template <typename T>
__global__ void trsm_left_kernel(const T *Lb, T *Zb, int bsp, int p) {
    __shared__ T L[PW][PW + 1];
    const T *A = Lb + (int64_t)blockIdx.x * bsp * bsp;
    T *Z = Zb + (int64_t)blockIdx.x * bsp * bsp;
    for (int e = threadIdx.x; e < PW * PW; e += blockDim.x) L[e / PW][e % PW] = A[(int64_t)(p + e / PW) * bsp + p + e % PW];
    __syncthreads();
    const int col = blockIdx.y * blockDim.x + threadIdx.x;
    if (col >= p + PW) return;
    T z[PW];
#pragma unroll
    for (int i = 0; i < PW; ++i) z[i] = Z[(int64_t)(p + i) * bsp + col];
#pragma unroll
    for (int i = 0; i < PW; ++i) {
        T s = z[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L[i][k] * z[k];
        z[i] = s / L[i][i];
    }
#pragma unroll
    for (int i = 0; i < PW; ++i) Z[(int64_t)(p + i) * bsp + col] = z[i];
}

template <typename T>
__global__ void identity_kernel(T *Zb, int bsp, int nb) {
    const int64_t tot = (int64_t)nb * bsp * bsp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % ((int64_t)bsp * bsp);
        Zb[e] = (r / bsp == r % bsp) ? T(1) : T(0);
    }
}

// The score pass of one block iteration, grid (blocks of rows, kScoreGroups column groups), 256
// threads per block of at most 1024 rows (four rows per thread):
//  * with Kd, first the residual update r -= K(X, X_blk) delta + sigma^2 delta on the selected
//    block's rows (Kd = K(X, X_blk) delta from the panel product);
//  * bpart[c][b] = sum over the block's rows of r_c^2 (the split norms' partials): each warp sums
//    its rows' squares per column by shuffles into its own shared-memory slot, the warps' slots
//    added in a fixed order at the end (FP64);
//  * rowsum[g][i] = sum of r_c[i] over the group's columns (the block score's row sums, in the
//    vectors' precision; ap_score_kernel adds the groups).
// The column groups put several CTAs on each block of rows, so that enough loads are in flight,
// and the loads of kCols columns are issued before their stores.  R <= 512.
constexpr int kScoreGroups = 8;
template <typename T>
__global__ void __launch_bounds__(256) ap_score_norm_kernel(T *r, int64_t n, int R, int bs, T *rowsum,
                                                            double *bpart, const SolverState *st, int skip_done,
                                                            const T *Kd, const T *delta, const int64_t *col0,
                                                            T sigma2) {
    if (skip_done && st->done) return;
    const int b = blockIdx.x, nb = gridDim.x, g = blockIdx.y;
    const int cpg = (R + (int)gridDim.y - 1) / (int)gridDim.y, cbeg = g * cpg, cend = min(R, cbeg + cpg);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t lo = (int64_t)b * bs, hi = min(n, lo + bs);
    const int64_t c0 = Kd ? *col0 : -1;
    constexpr int kRows = 4;  // rows per thread (bs <= 1024)
    constexpr int kCols = 2;  // columns whose loads are issued together (before any store)
    __shared__ T wsq[8][512];  // in the vectors' precision (FP32 squares of an FP64 residual underflow)
    T t[kRows];
#pragma unroll
    for (int k = 0; k < kRows; ++k) t[k] = T(0);
    for (int cb = cbeg; cb < cend; cb += kCols) {
        T x[kCols][kRows];
#pragma unroll
        for (int j = 0; j < kCols; ++j) {
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const int c = cb + j;
                const int64_t i = lo + threadIdx.x + (int64_t)k * blockDim.x;
                T v = T(0);
                if (c < cend && i < hi) {
                    v = r[(int64_t)c * n + i];
                    if (Kd) {
                        v -= Kd[(int64_t)c * n + i];
                        if (i >= c0 && i < c0 + bs) v -= sigma2 * delta[(int64_t)c * bs + (i - c0)];
                    }
                }
                x[j][k] = v;
            }
        }
#pragma unroll
        for (int j = 0; j < kCols; ++j) {
            const int c = cb + j;
            T sq = T(0);
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const int64_t i = lo + threadIdx.x + (int64_t)k * blockDim.x;
                if (Kd && c < cend && i < hi) r[(int64_t)c * n + i] = x[j][k];
                t[k] += x[j][k];
                sq += x[j][k] * x[j][k];
            }
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0 && c < cend) wsq[warp][c] = sq;
        }
    }
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        const int64_t i = lo + threadIdx.x + (int64_t)k * blockDim.x;
        if (i < hi) rowsum[(int64_t)g * n + i] = t[k];
    }
    __syncthreads();
    for (int c = cbeg + (int)threadIdx.x; c < cend; c += blockDim.x) {
        double a = 0.0;
        for (int w = 0; w < 8; ++w) a += (double)wsq[w][c];
        bpart[(int64_t)c * nb + b] = a;
    }
}

// Alg. 2's block score, score[b] = sum over the block's rows of (sum_g rowsum[g][i])^2 (the
// column groups added in order, FP64 squares).  One block of 256 threads per block of rows.
template <typename T>
__global__ void __launch_bounds__(256) ap_score_kernel(const T *rowsum, int64_t n, int bs, int G, double *score,
                                                       const SolverState *st, int skip_done) {
    if (skip_done && st->done) return;
    const int b = blockIdx.x;
    const int64_t lo = (int64_t)b * bs, hi = min(n, lo + bs);
    double s = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        T t = T(0);
        for (int g = 0; g < G; ++g) t += rowsum[(int64_t)g * n + i];
        s += (double)(t * t);
    }
    __shared__ double red[8];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
        score[b] = a;
    }
}

// argmax over blocks, ties to the lowest index; writes the row offset of the block.
__global__ void ap_select_kernel(const double *score, int nb, int bs, int64_t *col0, const SolverState *st) {
    if (st->done) return;
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    double best = -1.0;
    int besti = 0x7fffffff;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double v = score[b];
        if (v > best || (v == best && b < besti)) {
            best = v;
            besti = b;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            double v = bv[threadIdx.x + s];
            int i = bi[threadIdx.x + s];
            if (v > bv[threadIdx.x] || (v == bv[threadIdx.x] && i < bi[threadIdx.x])) {
                bv[threadIdx.x] = v;
                bi[threadIdx.x] = i;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *col0 = (int64_t)bi[0] * bs;
}

// Partial block solves: dpart[ks][c][a] = sum over the ks-th K range of Hinv[blk][a][a'] r[c][lo + a'],
// a < bs (rows beyond n -> 0).  grid (bs/64, R/16, kSplitK): the K ranges split the work over
// enough CTAs to fill the GPU (one 1024 x 1024 block against 65 vectors is 68M FMA).
constexpr int kSplitK = 8;
constexpr int kNormThreads = 1024;  // ap_norm_kernel's block
template <typename T>
__global__ void __launch_bounds__(256) ap_delta_kernel(const T *Hinv, int bsp, int bs, const T *r, int64_t n, int R,
                                                       const int64_t *col0, T *dpart, const SolverState *st) {
    if (st->done) return;
    __shared__ T Hs[64][33];
    __shared__ T Rs[32][17];
    const int64_t lo = *col0;
    const int blk = (int)(lo / bs);
    const int m = (int)min((int64_t)bs, n - lo);
    const T *Hm = Hinv + (int64_t)blk * bsp * bsp;
    const int a0 = blockIdx.x * 64, c0 = blockIdx.y * 16, ks = blockIdx.z;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int kper = (int)rup(cdiv(m, kSplitK), 32);
    const int kb = ks * kper, ke = min(m, kb + kper);
    T *delta = dpart + (int64_t)ks * R * bs;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int k0 = kb; k0 < ke; k0 += 32) {
        for (int e = tid; e < 64 * 32; e += 256) {
            int aa = e / 32, kk = e % 32;
            Hs[aa][kk] = (a0 + aa < m && k0 + kk < ke) ? Hm[(int64_t)(a0 + aa) * bsp + k0 + kk] : T(0);
        }
        for (int e = tid; e < 32 * 16; e += 256) {
            int cc = e / 32, kk = e % 32;
            Rs[kk][cc] = (k0 + kk < ke && c0 + cc < R) ? r[(int64_t)(c0 + cc) * n + lo + k0 + kk] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            T rv = Rs[kk][tx];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] += Hs[ty + 16 * i][kk] * rv;
        }
        __syncthreads();
    }
    const int c = c0 + tx;
    if (c >= R) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int a = a0 + ty + 16 * i;
        if (a < bs) delta[(int64_t)c * bs + a] = (a < m) ? acc[i] : T(0);
    }
}

// delta[c][a] = sum_ks dpart[ks][c][a] (K ranges in a fixed order); v[c][lo + a] += delta[c][a].
// With D16 (tensor-core panel, one block per column) also the panel product's fp16 operand:
// V16[c][a] = fp16(delta * 2^(1-e)) with max_a |delta[c][a]| = f 2^e, f in [0.5, 1), and
// vinv[c] = 2^(e-1) -- the product's own conversion rule, without its two launches.
template <typename T>
__global__ void __launch_bounds__(1024) ap_vupdate_kernel(T *V, int64_t n, int bs, int R, const int64_t *col0,
                                                         const T *dpart, T *delta, const SolverState *st,
                                                         __half *D16, int64_t p2, float *vinv) {
    if (st->done) return;
    const int c = blockIdx.y;
    const int64_t lo = *col0;
    const int m = (int)min((int64_t)bs, n - lo);
    float mx = 0.0f;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < bs; a += gridDim.x * blockDim.x) {
        T dl = T(0);
        for (int ks = 0; ks < kSplitK; ++ks) dl += dpart[((int64_t)ks * R + c) * bs + a];
        delta[(int64_t)c * bs + a] = dl;
        if (a < m) V[(int64_t)c * n + lo + a] += dl;
        mx = fmaxf(mx, fabsf((float)dl));
    }
    if constexpr (std::is_same<T, float>::value) {
        if (D16) {
            __shared__ float red[32];
            __shared__ float s_scale;
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
            __syncthreads();
            if (threadIdx.x == 0) {
                float t = 0.0f;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
                int e = 0;
                float scale = 1.0f, inv = 1.0f;
                if (t > 0.0f && isfinite(t)) {
                    frexpf(t, &e);
                    scale = ldexpf(1.0f, 1 - e);
                    inv = ldexpf(1.0f, e - 1);
                }
                s_scale = scale;
                vinv[c] = inv;
            }
            __syncthreads();
            const float sc = s_scale;
            // each thread converts the entries it has just written
            for (int a = threadIdx.x; a < bs; a += blockDim.x)
                D16[(int64_t)c * p2 + a] = __float2half_rn(delta[(int64_t)c * bs + a] * sc);
        }
    }
}

// Split norms and the loop condition from the ||r||^2 partials; the columns' sums in parallel (one
// warp per column; one thread per column summing its P partials in a dependent chain took
// ~27 us, a single thread for all R x P ~0.3 ms).  One block of kNormThreads.
__global__ void ap_norm_kernel(int R, int P, const double *part, SolverState *st, long long max_iters, double tol,
                               int stop_rule, int first) {
    if (!first && st->done) return;
    __shared__ double sq[512];
    // a warp per column: its P partials in one round of loads, then a fixed butterfly
    for (int c = (int)(threadIdx.x >> 5); c < R; c += (int)(blockDim.x >> 5)) {
        const double v = sum_parts_warp(part, c, P);
        if ((threadIdx.x & 31) == 0) sq[c] = v;
    }
    if (threadIdx.x == 0 && first) {
        st->done = 0;
        st->status = GP_OK;
    }
    __syncthreads();
    finish_norms_block(st, sq, R, first ? 0 : st->iter + 1, max_iters, tol, stop_rule);
    if (threadIdx.x == 0 && first == 2) st->certified = 1;  // the initial residual came from an exact-class product
}

}  // namespace

template <typename T>
static size_t ap_panel_ws(int64_t n, int64_t bs, int d, int R, int prec) {
    if (std::is_same<T, float>::value && prec == GP_PREC_TC16) {
        // tensor-core panel: all points prepared once per solve + the product's own scratch
        Carver c(nullptr);
        c.take<char>(tc_points_bytes(n, d));
        c.take<char>(tc_mvm_workspace(n, bs, R));
        return c.bytes();
    }
    return mvm_simt_workspace<T>(n, bs, R);
}

template <typename T>
size_t ap_workspace(int64_t n, int d, int R, int64_t bs, int prec) {
    const int P = nparts_for(n);
    const int64_t nb = cdiv(n, bs), bsp = rup(bs, PW);
    Carver c(nullptr);
    c.take<T>((size_t)R * n);               // residual
    c.take<T>((size_t)R * n);               // H v (set-up)
    c.take<T>((size_t)R * bs);              // delta
    c.take<T>((size_t)kSplitK * R * bs);    // partial block solves
    c.take<T>((size_t)nb * bsp * bsp);      // factor / inverse
    c.take<T>((size_t)nb * bsp * bsp);      // L^-1
    c.take<double>((size_t)R * P);
    c.take<double>((size_t)R);
    c.take<double>((size_t)nb);
    c.take<double>((size_t)R * nb);        // per-block partials of ||r_c||^2
    c.take<T>((size_t)kScoreGroups * n);   // the score's row sums per column group
    c.take<int64_t>(1);
    c.take<int>(1);
    c.take<SolverState>(1);
    c.take<char>(std::max(ap_panel_ws<T>(n, bs, d, R, prec), mvm_workspace<T>(n, n, d, R, prec)));
    if (std::is_same<T, float>::value && prec == GP_PREC_FP32) c.take<char>(f64_residual_workspace(n, d, R));
    if (std::is_same<T, float>::value && prec == GP_PREC_TC16 && R <= 128) {
        c.take<__half>((size_t)tc_rhs_pad(R) * tc_cols_pad(std::min<int64_t>(bs, n)));  // the update's fp16 operand
        c.take<float>(256);
    }
    return c.bytes();
}

template <typename T>
int ap_solve(const KP<T> &kp, const T *X, int64_t n, const T *B, int R, T *V, int64_t bs64, int64_t max_iters,
             double tol, int stop_rule, int prec, gp_solve_info_t *info, void *ws, size_t ws_bytes,
             cudaStream_t st) {
    if (R > 512) {
        set_error("nrhs must be <= 512");
        return GP_ERR_INVALID_ARG;
    }
    const int bs = (int)std::min<int64_t>(bs64, n);
    const int P = nparts_for(n);
    const int nb = (int)cdiv(n, bs);
    const int bsp = (int)rup(bs, PW);
    Carver c(ws);
    T *r = c.take<T>((size_t)R * n);
    T *HV = c.take<T>((size_t)R * n);
    T *delta = c.take<T>((size_t)R * bs);
    T *dpart = c.take<T>((size_t)kSplitK * R * bs);
    T *Hb = c.take<T>((size_t)nb * bsp * bsp);
    T *Zb = c.take<T>((size_t)nb * bsp * bsp);
    double *part = c.take<double>((size_t)R * P);
    double *scale = c.take<double>(R);
    double *score = c.take<double>(nb);
    double *bpart = c.take<double>((size_t)R * nb);
    T *rowsum = c.take<T>((size_t)kScoreGroups * n);
    int64_t *col0 = c.take<int64_t>(1);
    int *fail = c.take<int>(1);
    SolverState *sd = c.take<SolverState>(1);
    size_t mwb = std::max(ap_panel_ws<T>(n, bs, kp.d, R, prec), mvm_workspace<T>(n, n, kp.d, R, prec));
    void *mw = c.take<char>(mwb);
    const bool check64 = std::is_same<T, float>::value && prec == GP_PREC_FP32;
    const size_t c64b = check64 ? f64_residual_workspace(n, kp.d, R) : 0;
    void *c64w = check64 ? c.take<char>(c64b) : nullptr;
    // tensor-core panel: the block update kernel writes the product's fp16 operand itself
    const bool d16 = std::is_same<T, float>::value && prec == GP_PREC_TC16 && R <= 128;
    const int64_t p2b = tc_cols_pad(bs);
    __half *D16 = d16 ? c.take<__half>((size_t)tc_rhs_pad(R) * p2b) : nullptr;
    float *vinv16 = d16 ? c.take<float>(256) : nullptr;
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    if (d16) GP_TRY_CUDA(cudaMemsetAsync(D16, 0, sizeof(__half) * (size_t)tc_rhs_pad(R) * p2b, st));

    const dim3 gv((unsigned)std::min<int64_t>(cdiv(n, 2048), 1024), (unsigned)R);  // about 8 rows per thread
    const dim3 gp_((unsigned)P, (unsigned)R);
    // the true residual the tolerance is judged on: the tensor-core form's split product (the
    // initial residual uses the form's own product; the final check catches its error)
    const int prec_true = prec == GP_PREC_TC16 ? GP_PREC_TC16X3 : prec;
    // block scores and norm partials of the current residual; update: first apply the block
    // iteration's r -= K delta + sigma^2 delta (K delta in HV from the tensor-core panel)
    auto score_pass = [&](int skip_done, bool update) {
        ap_score_norm_kernel<T><<<dim3((unsigned)nb, kScoreGroups), 256, 0, st>>>(
            r, n, R, bs, rowsum, bpart, sd, skip_done, update ? HV : nullptr, delta, col0, kp.sigma2);
        ap_score_kernel<T><<<nb, 256, 0, st>>>(rowsum, n, bs, kScoreGroups, score, sd, skip_done);
    };
    const bool exact_start = !(std::is_same<T, float>::value && (prec == GP_PREC_TC16 || prec == GP_PREC_FP32));
    // ---- block inverses H[i,i]^-1 (cached for the whole solve)
    GP_TRY_CUDA(cudaMemsetAsync(fail, 0, sizeof(int), st));
    ap_build_blocks_kernel<T><<<dim3(bsp / 16, bsp / 16, nb), dim3(16, 16), 0, st>>>(kp, X, n, bs, bsp, Hb);
    GP_TRY(check_launch("ap_build_blocks_kernel", 1));
    for (int p = 0; p < bsp; p += PW) {
        potf2_kernel<T><<<nb, 32, 0, st>>>(Hb, bsp, p, fail);
        const int rest = bsp - p - PW;
        if (rest > 0) {
            trsm_right_kernel<T><<<dim3(nb, (unsigned)cdiv(rest, 128)), 128, 0, st>>>(Hb, bsp, p);
            const int64_t off = (int64_t)(p + PW) * bsp;
            // trailing update: only the lower triangle is read later
            GP_TRY((gemm_batched<T, false, true>(rest, rest, PW, T(-1), Hb + off + p, bsp, (int64_t)bsp * bsp,
                                                 Hb + off + p, bsp, (int64_t)bsp * bsp, T(1), Hb + off + p + PW, bsp,
                                                 (int64_t)bsp * bsp, nb, st, GemmShape{1, 0, 0})));
        }
        GP_TRY(check_launch("blocked cholesky", rest > 0 ? 2 : 1));
    }
    // L^-1 by blocked forward substitution on the identity
    identity_kernel<T><<<1024, 256, 0, st>>>(Zb, bsp, nb);
    GP_TRY(check_launch("identity_kernel"));
    for (int p = 0; p < bsp; p += PW) {
        if (p > 0)
            // Z[0:p, 0:p] is lower-triangular: column j of the product sums over k >= j
            GP_TRY((gemm_batched<T, false, false>(PW, p, p, T(-1), Hb + (int64_t)p * bsp, bsp, (int64_t)bsp * bsp, Zb,
                                                  bsp, (int64_t)bsp * bsp, T(1), Zb + (int64_t)p * bsp, bsp,
                                                  (int64_t)bsp * bsp, nb, st, GemmShape{0, 0, 1})));
        trsm_left_kernel<T><<<dim3(nb, (unsigned)cdiv(p + PW, 128)), 128, 0, st>>>(Hb, Zb, bsp, p);
        GP_TRY(check_launch("blocked triangular inverse"));
    }
    // H^-1 = L^-T L^-1
    // H^-1 = Z^T Z: symmetric, and (Z^T Z)_ij sums over k >= max(i, j) for the lower-triangular Z
    GP_TRY((gemm_batched<T, true, false>(bsp, bsp, bsp, T(1), Zb, bsp, (int64_t)bsp * bsp, Zb, bsp,
                                         (int64_t)bsp * bsp, T(0), Hb, bsp, (int64_t)bsp * bsp, nb, st,
                                         GemmShape{1, 1, 2})));

    // ---- normalisation and initial residual r = b~ - H v~
    coldot_kernel<T><<<gp_, 256, 0, st>>>(B, B, n, P, part, nullptr);
    norm_scale_kernel<<<1, 256, 0, st>>>(R, P, part, scale);
    scale_cols_kernel<T><<<gv, 256, 0, st>>>(V, n, scale, 1);
    GP_TRY(check_launch("ap setup", 3));
    GP_TRY(apply_mvm<T>(kp, X, n, X, n, V, n, R, HV, n, 1, prec, mw, mwb, st));
    init_residual_kernel<T><<<gv, 256, 0, st>>>(B, HV, r, (T *)nullptr, n, scale);
    score_pass(0, false);
    ap_norm_kernel<<<1, kNormThreads, 0, st>>>(R, nb, bpart, sd, (long long)max_iters, tol, stop_rule,
                                              exact_start ? 2 : 1);
    GP_TRY(check_launch("ap start", 4));

    int hfail = 0;
    GP_TRY_CUDA(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    SolverState hs{};
    GP_TRY(poll_state(sd, &hs, st));
    if (hfail) {
        scale_cols_kernel<T><<<gv, 256, 0, st>>>(V, n, scale, 0);
        set_error("AP: a diagonal block of H is not positive definite");
        GP_TRY_CUDA(cudaStreamSynchronize(st));
        info->status = GP_ERR_BREAKDOWN;
        return GP_ERR_BREAKDOWN;
    }
    MvmArgs<T> pa{};
    pa.kp = kp;
    pa.X1 = X;
    pa.n1 = n;
    pa.X2 = X;
    pa.n2 = bs;
    pa.n2_total = n;
    pa.col0_dev = col0;
    pa.V = delta;
    pa.ldv = bs;
    pa.R = R;
    pa.Y = r;
    pa.ldy = n;
    pa.alpha = T(-1);
    pa.beta = T(1);
    pa.diag_coef = -kp.sigma2;
    pa.Vd = delta;
    pa.ldvd = bs;
    pa.diag_from_col0 = 1;
    pa.done = &sd->done;
    // Tensor-core panel: K(X, X[col0 : col0 + bs]) over all points prepared once per solve
    // (after the initial residual, whose product used the same scratch), the block offset
    // read on the device.
    bool tc_panel = false;
    TcMvmArgs ta{};
    void *tw = nullptr, *pbuf = nullptr;
    size_t twb = 0;
    if constexpr (std::is_same<T, float>::value) {
        if (prec == GP_PREC_TC16) {
            tc_panel = true;
            Carver pc(mw);
            pbuf = pc.take<char>(tc_points_bytes(n, kp.d));
            twb = tc_mvm_workspace(n, bs, R);
            tw = pc.take<char>(twb);
            TcPoints pts;
            GP_TRY(tc_prepare_points(kp, X, n, pbuf, &pts, st));
            ta.kind = kp.kind;
            ta.rows = pts;
            ta.cols = pts;
            ta.ncols = bs;
            ta.col0_dev = col0;
            ta.diag_from_col0 = 1;
            // Kd = K(X, X_blk) delta into HV; the score kernel applies r -= Kd + sigma^2 delta (reading
            // the residual once there rather than in every row segment of the product's epilogue)
            ta.V = delta;
            ta.ldv = bs;
            ta.R = R;
            ta.Y = HV;
            ta.ldy = n;
            ta.sf2 = kp.sf2;
            ta.alpha = 1.0f;
            ta.beta = 0.0f;
            ta.diag_coef = 0.0f;
            ta.done = &sd->done;
            ta.V16pre = D16;  // written by the block update kernel (null: the product converts delta)
            ta.vinv_pre = vinv16;
        }
    }
    const dim3 gdel((unsigned)cdiv(bs, 64), (unsigned)cdiv(R, 16), (unsigned)kSplitK);
    // The residual of Alg. 2 is updated by the panel products (recursive); when the loop stops
    // on it, the true residual b~ - H v is recomputed (differences rounded once, FP64 norms) and replaces
    // it; the tolerance is judged on it, and a solve whose true residual misses the tolerance is
    // resumed within its budget, so the reported norms are true-residual norms.
    int64_t t = 0, chunk = 8;
    int checks = 0;
    double prev_y = 0.0, prev_z = 0.0;
    for (;;) {
    while (!hs.done && t < max_iters) {
        int64_t k = std::min<int64_t>(chunk, max_iters - t);
        for (int64_t it = 0; it < k; ++it, ++t) {
            // the scores of the current residual come from the previous pass over r
            ap_select_kernel<<<1, 1024, 0, st>>>(score, nb, bs, col0, sd);
            ap_delta_kernel<T><<<gdel, 256, 0, st>>>(Hb, bsp, bs, r, n, R, col0, dpart, sd);
            if (d16)
                ap_vupdate_kernel<T><<<dim3(1, R), 1024, 0, st>>>(V, n, bs, R, col0, dpart, delta, sd, D16, p2b, vinv16);
            else
                ap_vupdate_kernel<T><<<dim3((unsigned)cdiv(bs, 256), R), 256, 0, st>>>(V, n, bs, R, col0, dpart, delta,
                                                                                       sd, nullptr, 0, nullptr);
            GP_TRY(check_launch("ap iteration", 3));
            if constexpr (std::is_same<T, float>::value) {
                if (tc_panel) {
                    GP_TRY(tc_mvm(ta, tw, twb, st));
                } else {
                    GP_TRY(mvm_simt<T>(pa, mw, mwb, st));
                }
            } else {
                GP_TRY(mvm_simt<T>(pa, mw, mwb, st));
            }
            score_pass(1, tc_panel);
            ap_norm_kernel<<<1, kNormThreads, 0, st>>>(R, nb, bpart, sd, (long long)max_iters, tol, stop_rule, 0);
            GP_TRY(check_launch("ap norms", 3));
        }
        chunk = std::min<int64_t>(chunk * 2, 64);
        GP_TRY(poll_state(sd, &hs, st));
    }
    if (hs.status != GP_OK || hs.certified) break;
    // (the full product uses the scratch that holds the panel's prepared points; the FP32 form
    // takes the FP64 product, as gp_solve_cg does)
    if (check64) {
        if constexpr (std::is_same<T, float>::value)
            GP_TRY(f64_residual(kp, X, n, B, V, R, scale, r, part, P, c64w, c64b, st));
    } else {
        GP_TRY(apply_mvm<T>(kp, X, n, X, n, V, n, R, HV, n, 1, prec_true, mw, mwb, st));
        true_residual_kernel<T, T><<<gp_, 256, 0, st>>>(B, HV, r, n, P, scale, part, nullptr);
    }
    true_state_kernel<<<1, 256, 0, st>>>(R, P, nullptr, part, nullptr, sd, (long long)max_iters, tol, stop_rule, 1);
    // the block scores of the replaced residual (for the next selection; its norms are set)
    score_pass(0, false);
    GP_TRY(check_launch("ap true residual", 4));
    GP_TRY(poll_state(sd, &hs, st));
    t = hs.iter;
    if (hs.done) break;
    // a resumed solve whose true residual did not fall by 10% since the previous check has
    // reached the accuracy its arithmetic attains: stop there, not converged
    if (checks > 0 && std::max(hs.res_y / prev_y, hs.res_z / prev_z) > 0.9) break;
    prev_y = hs.res_y;
    prev_z = hs.res_z;
    ++checks;
    if constexpr (std::is_same<T, float>::value) {
        if (tc_panel) {
            TcPoints pts;
            GP_TRY(tc_prepare_points(kp, X, n, pbuf, &pts, st));
        }
    }
    chunk = 4;
    }
    scale_cols_kernel<T><<<gv, 256, 0, st>>>(V, n, scale, 0);
    GP_TRY(check_launch("ap rescale"));
    GP_TRY(poll_state(sd, &hs, st));
    fill_info(hs, info);
    if (hs.status != GP_OK) {
        set_error("AP breakdown at iteration %lld", hs.iter);
        return hs.status;
    }
    return GP_OK;
}

template size_t ap_workspace<float>(int64_t, int, int, int64_t, int);
template size_t ap_workspace<double>(int64_t, int, int, int64_t, int);
template int ap_solve<float>(const KP<float> &, const float *, int64_t, const float *, int, float *, int64_t,
                             int64_t, double, int, int, gp_solve_info_t *, void *, size_t, cudaStream_t);
template int ap_solve<double>(const KP<double> &, const double *, int64_t, const double *, int, double *, int64_t,
                              int64_t, double, int, int, gp_solve_info_t *, void *, size_t, cudaStream_t);

}  // namespace gp
