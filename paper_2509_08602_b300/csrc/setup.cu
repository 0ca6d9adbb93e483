// Case set-up on the device: dual-LP assembly (Appendix A), row and BOT-column
// scaling (Sec. 3.C), rounding of A for the iterations, S = A A^T + I in FP64,
// its FP64 Cholesky factor and the explicit inverse kept for the iterations
// (Sec. 2.B caches a factorisation; Sec. 3.A keeps the explicit inverse).
#include <math.h>

#include <algorithm>
#include <cfloat>
#include <string>
#include <vector>

#include "lgk_impl.hpp"

namespace lgk {

int DevBuf::alloc(size_t n) {
    if (p) { cudaFree(p); p = nullptr; bytes = 0; }
    if (n == 0) return LGK_OK;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc(" + std::to_string(n) + " bytes): " + cudaGetErrorString(e));
        return LGK_ENOMEM;
    }
    bytes = n;
    return LGK_OK;
}

size_t CaseData::bytes_held() const {
    return col_slot.bytes + Dr.bytes + A32.bytes + Ahat.bytes + G32.bytes + G3.bytes + S3.bytes +
           cublas_ws.bytes + ctrl_setup.bytes;
}

// ------------------------------------------------------------- assembly

// A[b][p] = sign_p phi[p][b] / D_p for point columns (32x32 tiled transpose).
// phi is validated here, on its one pass through the device: an entry that is
// negative, infinite or NaN sets *bad.
__global__ void k_assemble_points(const double* __restrict__ phi, const double* __restrict__ scale,
                                  int P, int B, double* __restrict__ A, int lda, int* bad) {
    __shared__ double tile[32][33];
    int p0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        int p = p0 + k, b = b0 + threadIdx.x;
        double v = 0.0;
        if (p < P && b < B) {
            v = phi[(size_t)p * B + b];
            if (!(v >= 0.0 && v <= DBL_MAX)) atomicExch(bad, 1);
        }
        tile[k][threadIdx.x] = v * (p < P ? scale[p] : 0.0);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        int b = b0 + k, p = p0 + threadIdx.x;
        if (b < B && p < P) A[(size_t)b * lda + p] = tile[threadIdx.x][k];
    }
}

// BOT columns p = P + (8 i + s): -C_S^T on beam rows (i, s, *), T^T on row B + i.
__global__ void k_assemble_bot(int P, int n_iso, int B, double cs, double* __restrict__ A, int lda) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;     // (iso, sector) pair
    if (q >= 8 * n_iso) return;
    int col = P + q;
    for (int c = 0; c < 3; ++c) A[(size_t)(3 * q + c) * lda + col] = -cs;
    A[(size_t)(B + q / 8) * lda + col] = 1.0;
}

// D_r[i] = 1 / ||A[i, :]||_2 (1 for empty rows).  One block per row, fixed
// reduction order (deterministic).
__global__ void k_row_norm(const double* __restrict__ A, int lda, int ncols, int m,
                           double* __restrict__ Dr) {
    int i = blockIdx.x;
    __shared__ double red[256];
    double s = 0.0;
    if (i < m)
        for (int p = threadIdx.x; p < ncols; p += 256) {
            double a = A[(size_t)i * lda + p];
            s += a * a;
        }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) Dr[i] = (i < m && red[0] > 0.0) ? 1.0 / sqrt(red[0]) : 1.0;
}

// Scale rows by D_r and the BOT columns [P, n) by beta, round for the
// iterations, and keep the rounded value in FP64 for S.  BF16 forms: NA terms
// hi (+ lo), each the BF16 rounding of what the earlier terms leave, so
// A = hi + lo holds exactly in FP64.
template <int NA>
__global__ void k_scale_round(double* __restrict__ A64, const double* __restrict__ Dr, int m_pad,
                              int n_pad, int P, int n, double beta, void* __restrict__ out, int keep) {
    const size_t total = (size_t)m_pad * n_pad;
    // rows over blockIdx.y (grid-stride), columns over x: no 64-bit division
    for (int i = blockIdx.y; i < m_pad; i += gridDim.y)
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += gridDim.x * blockDim.x) {
        const size_t e = (size_t)i * n_pad + p;
        double a = A64[e] * Dr[i];
        if (p >= P && p < n) a *= beta;
        if (NA > 0) {
            __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out);
            __nv_bfloat16 h = bf16_from_double(a);
            double kept = (double)__bfloat162float(h);
            o[e] = h;
            if (NA > 1) {
                __nv_bfloat16 l = bf16_from_double(a - kept);
                o[total + e] = l;
                kept += (double)__bfloat162float(l);
            }
            if (keep) A64[e] = kept;
        } else {
            float f = (float)a;
            static_cast<float*>(out)[e] = f;
            if (keep) A64[e] = (double)f;
        }
    }
}

// ---------------------------------------------------------------- FP64 GEMM
// C[M x N] = alpha op(A) op(B) + beta C; op(A) M x K (TA: A stored K x M),
// op(B) K x N (TB: B stored N x K).  LOWER skips tiles above the diagonal.
// TRI (C = Y^T Y with Y lower triangular, stored K x M and K x N): the terms
// k < max(row, column) are zero, so a tile's k range starts at the larger of
// its first row and column.
template <bool TA, bool TB, bool LOWER, bool TRI = false>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha,
                                               const double* __restrict__ A, int lda,
                                               const double* __restrict__ B, int ldb,
                                               double beta, double* __restrict__ C, int ldc) {
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    int tm = blockIdx.y, tn = blockIdx.x;
    if (LOWER && tn > tm) return;
    int m0 = tm * 64, n0 = tn * 64;
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = TRI ? max(m0, n0) : 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int mm, kk;
            if (TA) { kk = e >> 6; mm = e & 63; } else { mm = e >> 4; kk = e & 15; }
            int gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < K) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int nn, kk;
            if (TB) { nn = e >> 4; kk = e & 15; } else { kk = e >> 6; nn = e & 63; }
            int gn = n0 + nn, gk = k0 + kk;
            double v = 0.0;
            if (gn < N && gk < K) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
            if (gm < M && gn < N) {
                size_t o = (size_t)gm * ldc + gn;
                C[o] = alpha * acc[i][j] + (beta != 0.0 ? beta * C[o] : 0.0);
            }
        }
}

int dgemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
          int lda, const double* B, int ldb, double beta, double* C, int ldc) {
    if (M <= 0 || N <= 0) return LGK_OK;
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    if (!ta && !tb) k_dgemm<false, false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (!ta && tb) k_dgemm<false, true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (ta && !tb) k_dgemm<true, false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else k_dgemm<true, true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    LGK_LAUNCH_CHECK();
    return LGK_OK;
}

static int dgemm_lower_nt(cudaStream_t st, int M, int K, double alpha, const double* A, int lda,
                          double beta, double* C, int ldc) {
    if (M <= 0) return LGK_OK;
    dim3 grid((M + 63) / 64, (M + 63) / 64);
    k_dgemm<false, true, true><<<grid, 256, 0, st>>>(M, M, K, alpha, A, lda, A, lda, beta, C, ldc);
    LGK_LAUNCH_CHECK();
    return LGK_OK;
}

__global__ void k_add_identity(double* S, int ld, int m) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) S[(size_t)i * ld + i] += 1.0;
}

// ------------------------------------------------------------ FP64 Cholesky
constexpr int NB = 64;

// Factor the diagonal block at (k0, k0) in place: lower triangle <- L_kk.
__global__ void k_potrf_diag(double* S, int ld, int k0, int* err) {
    __shared__ double T[NB][NB + 1];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        int i = e / NB, j = e % NB;
        T[i][j] = S[(size_t)(k0 + i) * ld + k0 + j];
    }
    __syncthreads();
    for (int j = 0; j < NB; ++j) {
        if (threadIdx.x == 0) {
            double d = T[j][j];
            if (!(d > 0.0)) { atomicExch(err, DERR_NOT_PD); d = 1.0; }
            T[j][j] = sqrt(d);
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < NB; i += blockDim.x) T[i][j] /= T[j][j];
        __syncthreads();
        int w = NB - 1 - j;     // trailing (i, k) with j < k <= i < NB
        for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
            int i = j + 1 + e / w, k = j + 1 + e % w;
            if (k <= i) T[i][k] -= T[i][j] * T[k][j];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        int i = e / NB, j = e % NB;
        S[(size_t)(k0 + i) * ld + k0 + j] = (j <= i) ? T[i][j] : 0.0;
    }
}

// Rows r >= k0 + NB of the block column: L[r, k0:k0+NB] = S[r, k0:k0+NB] L_kk^{-T}.
__global__ void k_trsm_panel(double* S, int ld, int k0, int M) {
    __shared__ double Lk[NB][NB + 1];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        int i = e / NB, j = e % NB;
        Lk[i][j] = S[(size_t)(k0 + i) * ld + k0 + j];
    }
    __syncthreads();
    int r = k0 + NB + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    double* row = S + (size_t)r * ld + k0;
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) x[j] = row[j];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        double s = x[j];
#pragma unroll
        for (int t = 0; t < j; ++t) s -= x[t] * Lk[j][t];
        x[j] = s / Lk[j][j];
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) row[j] = x[j];
}

// Zero the strict upper triangle (leaves L alone in the buffer).
__global__ void k_zero_upper(double* S, int ld, int m) {
    size_t total = (size_t)m * m;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e / m), j = (int)(e % m);
        if (j > i) S[(size_t)i * ld + j] = 0.0;
    }
}

__global__ void k_set_identity(double* Y, int ld, int m) {
    size_t total = (size_t)m * m;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e / m), j = (int)(e % m);
        Y[(size_t)i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
}

// Y[k0:k0+NB, c] <- L_kk^{-1} Y[k0:k0+NB, c] for columns c < ncols.
__global__ void k_trsm_rows(const double* L, int ldl, double* Y, int ldy, int k0, int ncols) {
    __shared__ double Lk[NB][NB + 1];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        int i = e / NB, j = e % NB;
        Lk[i][j] = L[(size_t)(k0 + i) * ldl + k0 + j];
    }
    __syncthreads();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) x[j] = Y[(size_t)(k0 + j) * ldy + c];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        double s = x[j];
#pragma unroll
        for (int t = 0; t < j; ++t) s -= Lk[j][t] * x[t];
        x[j] = s / Lk[j][j];
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) Y[(size_t)(k0 + j) * ldy + c] = x[j];
}

// S^{-1} -> FP32, or -> three BF16 terms hi + mid + lo (each the bf16
// rounding of what the previous terms leave).
__global__ void k_inverse_out(const double* G, size_t total, float* g32, __nv_bfloat16* g3) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        double g = G[e];
        if (g32) g32[e] = (float)g;
        if (g3) {
            __nv_bfloat16 h = bf16_from_double(g);
            double r1 = g - (double)__bfloat162float(h);
            __nv_bfloat16 mid = bf16_from_double(r1);
            double r2 = r1 - (double)__bfloat162float(mid);
            g3[e] = h;
            g3[total + e] = mid;
            g3[2 * total + e] = bf16_from_double(r2);
        }
    }
}

// S (lower triangle computed, FP64) -> three BF16 terms of the full symmetric
// matrix, hi + mid + lo, for the solve's refinement (S v in the residual).
__global__ void k_split3_sym(const double* S, int ld, int m, __nv_bfloat16* s3) {
    const size_t total = (size_t)m * m;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / m), j = (int)(e % m);
        const double g = j <= i ? S[(size_t)i * ld + j] : S[(size_t)j * ld + i];
        __nv_bfloat16 h = bf16_from_double(g);
        const double r1 = g - (double)__bfloat162float(h);
        __nv_bfloat16 mid = bf16_from_double(r1);
        const double r2 = r1 - (double)__bfloat162float(mid);
        s3[e] = h;
        s3[total + e] = mid;
        s3[2 * total + e] = bf16_from_double(r2);
    }
}

// S[i][j] = S[j][i] for j > i: the upper triangle from the lower one (32 x 32
// tiles through shared memory, so both sides are read and written in rows).
__global__ void k_mirror_lower(double* S, int ld, int m) {
    __shared__ double t[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;       // destination tile (rows bi, cols bj), bj >= bi
    if (bj < bi) return;
    const int tx = threadIdx.x, ty = threadIdx.y;     // 32 x 8 threads
    for (int k = ty; k < 32; k += 8) {                // source tile (rows bj, cols bi)
        const int r = bj * 32 + k, c = bi * 32 + tx;
        t[k][tx] = (r < m && c < m) ? S[(size_t)r * ld + c] : 0.0;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int r = bi * 32 + k, c = bj * 32 + tx;
        if (r < m && c < m && c > r) S[(size_t)r * ld + c] = t[tx][k];
    }
}

// y = S x (S full, FP64), one warp per row, fixed summation order.
__global__ void k_symv(const double* __restrict__ S, int ld, int m, const double* __restrict__ x, double* y) {
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= m) return;
    double s = 0.0;
    for (int j = lane; j < m; j += 32) s += S[(size_t)row * ld + j] * x[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
}

// out[0] = x . y, out[1] = y . y (one block, fixed order)
__global__ void k_dot2(const double* x, const double* y, int m, double* out) {
    __shared__ double a[256], b[256];
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < m; i += 256) {
        sa += x[i] * y[i];
        sb += y[i] * y[i];
    }
    a[threadIdx.x] = sa;
    b[threadIdx.x] = sb;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            a[threadIdx.x] += a[threadIdx.x + w];
            b[threadIdx.x] += b[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = a[0];
        out[1] = b[0];
    }
}

__global__ void k_scale_vec(const double* y, int m, const double* nrm2, double* x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) x[i] = y[i] / sqrt(nrm2[1]);
}

__global__ void k_fill(double* x, int m, double v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) x[i] = v;
}

// ||A||_2 from S = I + A A^T: power iteration on S (S's entries are mostly
// positive, so the all-ones start overlaps its top eigenvector), Rayleigh
// quotient lambda_max(S) = 1 + ||A||_2^2.  S must be full (mirrored).
static int a_norm_estimate(cudaStream_t st, const double* S, int ld, int m, double* out) {
    DevBuf x, y, d;
    int rc;
    if ((rc = x.alloc((size_t)m * 8)) || (rc = y.alloc((size_t)m * 8)) || (rc = d.alloc(16))) return rc;
    const int g = (m + 255) / 256;
    k_fill<<<g, 256, 0, st>>>(x.as<double>(), m, 1.0 / sqrt((double)m));
    LGK_LAUNCH_CHECK();
    double h[2] = {0.0, 0.0};
    for (int it = 0; it < 60; ++it) {
        k_symv<<<(m + 7) / 8, 256, 0, st>>>(S, ld, m, x.as<double>(), y.as<double>());
        LGK_LAUNCH_CHECK();
        k_dot2<<<1, 256, 0, st>>>(x.as<double>(), y.as<double>(), m, d.as<double>());
        LGK_LAUNCH_CHECK();
        k_scale_vec<<<g, 256, 0, st>>>(y.as<double>(), m, d.as<double>(), x.as<double>());
        LGK_LAUNCH_CHECK();
    }
    LGK_CUDA_TRY(cudaMemcpyAsync(h, d.p, 16, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    *out = sqrt(std::max(h[0] - 1.0, 0.0));      // x . S x with ||x|| = 1
    return LGK_OK;
}

// ----------------------------------------------------------------- set-up

int setup_case(CaseData& cs, const lgk_case_desc& d) {
    cudaStream_t st = cs.stream;
    const int P = d.n_pts, N = d.n_iso, B = 24 * N;
    const int m = B + N, n = P + 8 * N;
    // multiples of 256: the GEMMs may run 256-row tiles over either dimension
    const int m_pad = (int)round_up(m, 256), n_pad = (int)round_up(n, 256);
    const int T = d.n_targets;
    cs.n_iso = N; cs.n_pts = P; cs.n_beams = B; cs.m = m; cs.n = n;
    cs.m_pad = m_pad; cs.n_pad = n_pad;
    cs.n_targets = T; cs.n_oars = d.n_oars; cs.n_slot = n_slots(T);
    const bool bf16 = cs.prm.precision != LGK_PREC_FP32;
    cs.na = cs.prm.precision == LGK_PREC_BF16X3 ? 2 : (bf16 ? 1 : 0);

    // resident footprint check before any large allocation
    size_t resident = (size_t)n_pad + (size_t)m_pad * 8 + 64 +
                      (bf16 ? (size_t)cs.na * m_pad * n_pad * 2 +
                                  (size_t)(keeps_s3(cs.prm) ? 6 : 3) * m_pad * m_pad * 2
                            : (size_t)m_pad * n_pad * 4 + (size_t)m_pad * m_pad * 4);
    if (cs.prm.hbm_budget && resident > cs.prm.hbm_budget) {
        set_error("case footprint " + std::to_string(resident) + " B exceeds hbm_budget " +
                  std::to_string(cs.prm.hbm_budget) + " B");
        return LGK_EBUDGET;
    }

    // per-point slot, threshold and sign (Appendix A)
    std::vector<uint8_t> slot(n_pad, (uint8_t)slot_pad(T));
    std::vector<double> scale(P);
    cs.slot_count.assign(cs.n_slot, 0);
    double d_mean = 0.0;
    for (int k = 0; k < T; ++k) d_mean += d.d_presc[k];
    d_mean /= T;
    for (int p = 0; p < P; ++p) {
        int k = d.kind[p], s = d.struct_id[p];
        int sl;
        double D, sign;
        switch (k) {
            case LGK_TS: sl = 3 * s; D = d.d_presc[s]; sign = 1.0; break;
            case LGK_TI: sl = 3 * s + 1; D = d.d_presc[s]; sign = 1.0; break;
            case LGK_R: sl = 3 * s + 2; D = d.d_presc[s]; sign = -1.0; break;
            case LGK_LD1: sl = slot_ld1(T); D = d.d_ld1; sign = -1.0; break;
            case LGK_LD2: sl = slot_ld2(T); D = d.d_ld2; sign = -1.0; break;
            default: sl = slot_oar(T); D = d.d_oar[s]; sign = -1.0; break;
        }
        slot[p] = (uint8_t)sl;
        scale[p] = sign / D;
        cs.slot_count[sl] += 1;
    }
    cs.slot_host.assign(slot.begin(), slot.begin() + P);
    for (int q = P; q < n; ++q) slot[q] = (uint8_t)slot_bot(T);
    cs.c_of_slot.assign(cs.n_slot, 0.0f);
    for (int k = 0; k < T; ++k) {
        cs.c_of_slot[3 * k] = -1.0f;
        cs.c_of_slot[3 * k + 1] = -1.0f;
        cs.c_of_slot[3 * k + 2] = 1.0f;
    }
    cs.c_of_slot[slot_ld1(T)] = 1.0f;
    cs.c_of_slot[slot_ld2(T)] = 1.0f;
    cs.c_of_slot[slot_oar(T)] = 1.0f;
    cs.q_area.assign(d.q_area, d.q_area + T);
    cs.q_vol.assign(d.q_vol, d.q_vol + T);
    cs.d_presc.assign(d.d_presc, d.d_presc + T);
    int n_cost = 0;
    for (int p = 0; p < P; ++p) n_cost += d.kind[p] != LGK_OAR;
    cs.beta = cs.prm.scale_bot ? n_cost / 2000.0 : 1.0;

    int rc;
    if ((rc = cs.col_slot.alloc(n_pad))) return rc;
    if ((rc = cs.Dr.alloc((size_t)m_pad * 8))) return rc;
    if ((rc = cs.ctrl_setup.alloc(16))) return rc;
    LGK_CUDA_TRY(cudaMemcpyAsync(cs.col_slot.p, slot.data(), n_pad, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemsetAsync(cs.ctrl_setup.p, 0, 16, st));

    // ---- A in FP64 (temporary)
    DevBuf A64, phi_d, scale_d;
    if ((rc = A64.alloc((size_t)m_pad * n_pad * 8))) return rc;
    if ((rc = phi_d.alloc((size_t)P * B * 8))) return rc;
    if ((rc = scale_d.alloc((size_t)P * 8))) return rc;
    LGK_CUDA_TRY(cudaMemsetAsync(A64.p, 0, A64.bytes, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(phi_d.p, d.phi, phi_d.bytes, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(scale_d.p, scale.data(), scale_d.bytes, cudaMemcpyHostToDevice, st));
    {
        dim3 grid((P + 31) / 32, (B + 31) / 32), blk(32, 8);
        k_assemble_points<<<grid, blk, 0, st>>>(phi_d.as<double>(), scale_d.as<double>(), P, B,
                                                A64.as<double>(), n_pad, cs.ctrl_setup.as<int>() + 1);
        LGK_LAUNCH_CHECK();
        k_assemble_bot<<<(8 * N + 255) / 256, 256, 0, st>>>(P, N, B, d.phi_cal / d_mean,
                                                            A64.as<double>(), n_pad);
        LGK_LAUNCH_CHECK();
    }
    {
        int bad = 0;
        LGK_CUDA_TRY(cudaMemcpyAsync(&bad, cs.ctrl_setup.as<int>() + 1, 4, cudaMemcpyDeviceToHost, st));
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
        if (bad) {
            set_error("phi must be finite and >= 0");
            return LGK_EINVAL;
        }
    }
    phi_d.alloc(0);
    scale_d.alloc(0);

    // ---- row norms, scaling, rounding (Sec. 3.C)
    if (cs.prm.normalize_rows) {
        k_row_norm<<<m_pad, 256, 0, st>>>(A64.as<double>(), n_pad, n_pad, m, cs.Dr.as<double>());
        LGK_LAUNCH_CHECK();
    } else {
        std::vector<double> ones(m_pad, 1.0);
        LGK_CUDA_TRY(cudaMemcpyAsync(cs.Dr.p, ones.data(), (size_t)m_pad * 8, cudaMemcpyHostToDevice, st));
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // ---- S = A A^T + I from exactly the rounded A, Cholesky, inverse.  BF16
    // forms: on the tensor cores from the BF16 terms (exact products, FP32
    // sums of short chunks, FP64 across chunks); FP32 form, or setup_fp64:
    // FP64 products on the CUDA cores (from the FP64 copy of the rounded A,
    // which only then is written back).
    DevBuf S, Y;
    const bool tc_s = bf16 && !cs.prm.setup_fp64;
    {
        const dim3 grid(8, (unsigned)std::min(m_pad, 4096));
        const int keep = tc_s ? 0 : 1;
        if (cs.na == 2) {
            if ((rc = cs.Ahat.alloc((size_t)2 * m_pad * n_pad * 2))) return rc;
            k_scale_round<2><<<grid, 256, 0, st>>>(A64.as<double>(), cs.Dr.as<double>(), m_pad, n_pad, P, n,
                                                   cs.beta, cs.Ahat.p, keep);
        } else if (cs.na == 1) {
            if ((rc = cs.Ahat.alloc((size_t)m_pad * n_pad * 2))) return rc;
            k_scale_round<1><<<grid, 256, 0, st>>>(A64.as<double>(), cs.Dr.as<double>(), m_pad, n_pad, P, n,
                                                   cs.beta, cs.Ahat.p, keep);
        } else {
            if ((rc = cs.A32.alloc((size_t)m_pad * n_pad * 4))) return rc;
            k_scale_round<0><<<grid, 256, 0, st>>>(A64.as<double>(), cs.Dr.as<double>(), m_pad, n_pad, P, n,
                                                   cs.beta, cs.A32.p, keep);
        }
        LGK_LAUNCH_CHECK();
    }
    if (tc_s) {
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
        A64.alloc(0);               // the BF16 terms are all the tensor cores need
    }
    if ((rc = S.alloc((size_t)m_pad * m_pad * 8))) return rc;
    if (tc_s) {
        if ((rc = tc_syrk(cs, S.as<double>(), cs.ctrl_setup.as<int>()))) return rc;
        int e0 = 0;
        LGK_CUDA_TRY(cudaMemcpy(&e0, cs.ctrl_setup.p, 4, cudaMemcpyDeviceToHost));
        if (e0) {
            set_error("tensor-core S = A A^T + I: device error flag " + std::to_string(e0));
            return LGK_ECUDA;
        }
    } else {
        if ((rc = dgemm_lower_nt(st, m_pad, n_pad, 1.0, A64.as<double>(), n_pad, 0.0, S.as<double>(), m_pad)))
            return rc;
        k_add_identity<<<(m_pad + 255) / 256, 256, 0, st>>>(S.as<double>(), m_pad, m_pad);
        LGK_LAUNCH_CHECK();
    }
    {
        // ||A||_2 (the FP64 plan check bounds a converged plan's constraint
        // violation by (1 + ||A||_2) tol ||z||)
        dim3 gt((m_pad + 31) / 32, (m_pad + 31) / 32), bt(32, 8);
        k_mirror_lower<<<gt, bt, 0, st>>>(S.as<double>(), m_pad, m_pad);
        LGK_LAUNCH_CHECK();
        if ((rc = a_norm_estimate(st, S.as<double>(), m_pad, m_pad, &cs.a_norm))) return rc;
    }
    if (bf16 && keeps_s3(cs.prm)) {     // S itself, for the refinement's residual rhs - S v
        if ((rc = cs.S3.alloc((size_t)m_pad * m_pad * 3 * 2))) return rc;
        k_split3_sym<<<148 * 8, 256, 0, st>>>(S.as<double>(), m_pad, m_pad, cs.S3.as<__nv_bfloat16>());
        LGK_LAUNCH_CHECK();
    }
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    A64.alloc(0);

    double* Sd = S.as<double>();
    int* err = cs.ctrl_setup.as<int>();
    for (int k0 = 0; k0 < m_pad; k0 += NB) {
        k_potrf_diag<<<1, 256, 0, st>>>(Sd, m_pad, k0, err);
        LGK_LAUNCH_CHECK();
        int rows = m_pad - k0 - NB;
        if (rows > 0) {
            k_trsm_panel<<<(rows + 127) / 128, 128, 0, st>>>(Sd, m_pad, k0, m_pad);
            LGK_LAUNCH_CHECK();
            double* panel = Sd + (size_t)(k0 + NB) * m_pad + k0;
            double* trail = Sd + (size_t)(k0 + NB) * m_pad + k0 + NB;
            if ((rc = dgemm_lower_nt(st, rows, NB, -1.0, panel, m_pad, 1.0, trail, m_pad))) return rc;
        }
    }
    k_zero_upper<<<148 * 8, 256, 0, st>>>(Sd, m_pad, m_pad);
    LGK_LAUNCH_CHECK();
    int h_err = 0;
    LGK_CUDA_TRY(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err == DERR_NOT_PD) {
        set_error("S = A A^T + I is not positive definite in FP64 (Cholesky pivot <= 0)");
        return LGK_ENOTPD;
    }
    // Y = L^{-1} by blocked forward substitution on the identity
    if ((rc = Y.alloc((size_t)m_pad * m_pad * 8))) return rc;
    double* Yd = Y.as<double>();
    k_set_identity<<<148 * 8, 256, 0, st>>>(Yd, m_pad, m_pad);
    LGK_LAUNCH_CHECK();
    for (int k0 = 0; k0 < m_pad; k0 += NB) {
        int ncols = k0 + NB;
        k_trsm_rows<<<(ncols + 127) / 128, 128, 0, st>>>(Sd, m_pad, Yd, m_pad, k0, ncols);
        LGK_LAUNCH_CHECK();
        int rows = m_pad - k0 - NB;
        if (rows > 0) {
            if ((rc = dgemm(st, false, false, rows, ncols, NB, -1.0, Sd + (size_t)(k0 + NB) * m_pad + k0,
                            m_pad, Yd + (size_t)k0 * m_pad, m_pad, 1.0, Yd + (size_t)(k0 + NB) * m_pad,
                            m_pad)))
                return rc;
        }
    }
    // S^{-1} = L^{-T} L^{-1} = Y^T Y (reuse the S buffer): the lower tiles,
    // each over its k range (Y lower triangular: a sixth of the full
    // product's flops), then the upper triangle mirrored from the lower
    {
        dim3 grid((m_pad + 63) / 64, (m_pad + 63) / 64);
        k_dgemm<true, false, true, true><<<grid, 256, 0, st>>>(m_pad, m_pad, m_pad, 1.0, Yd, m_pad, Yd, m_pad,
                                                               0.0, Sd, m_pad);
        LGK_LAUNCH_CHECK();
        dim3 gt((m_pad + 31) / 32, (m_pad + 31) / 32), bt(32, 8);
        k_mirror_lower<<<gt, bt, 0, st>>>(Sd, m_pad, m_pad);
        LGK_LAUNCH_CHECK();
    }
    size_t mm = (size_t)m_pad * m_pad;
    if (bf16) {
        if ((rc = cs.G3.alloc(mm * 3 * 2))) return rc;
        k_inverse_out<<<148 * 8, 256, 0, st>>>(Sd, mm, nullptr, cs.G3.as<__nv_bfloat16>());
    } else {
        if ((rc = cs.G32.alloc(mm * 4))) return rc;
        k_inverse_out<<<148 * 8, 256, 0, st>>>(Sd, mm, cs.G32.as<float>(), nullptr);
    }
    LGK_LAUNCH_CHECK();
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    return LGK_OK;
}

}  // namespace lgk
