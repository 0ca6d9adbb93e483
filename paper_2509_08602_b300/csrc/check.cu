// FP64 check of finished plans (Sec. 2.B: the primal solution is recovered
// from the scaled multipliers rho y2; the LP it came from is Eq. dual_problem
// with the bounds of Appendix A).
//
// The iterations run in BF16/FP32 arithmetic and their stop test uses FP32
// partial sums.  This pass re-evaluates each finished column in FP64 from the
// state the library reports, against the exact LP (bounds u and b in FP64):
//   z1  = clip(q1, 0, u)        the dual LP's variables (what c^T z1 uses)
//   lam = rho max(q2 - b, 0)    the scaled multipliers (sector and isocenter
//                               times before the row scale)
// and computes, with A the matrix the iterations use (its BF16 terms summed
// in FP64, or the FP32 copy):
//   obj       c^T z1
//   plan      b^T lam + sum over finite-u columns of u (-(c + A^T lam))_+
//             (the weighted-sum objective of Sec. 2.A at the multipliers:
//             the LP dual's objective is -plan)
//   gap       (obj + plan) / max(1, |obj|)   duality gap, relative
//   infeas    ||(A z1 - b)_+||_2 / || |A| z1 ||_2   normwise backward error of
//             A z1 <= b: the constraint rows cancel large terms, so the
//             violation is measured against the size of those terms
//   infeas_abs ||(A z1 - b)_+||_2
//   hard      max over u = inf columns of (-(c + A^T lam))_+ / max lam
//             (organ limits and the BOT coupling, Appendix A)
//   bound     max over finite-u columns of (z1 - u)_+ (the iterations clip
//             to FP32 bounds)
// A z1 and A^T lam are FP64 dot products (|A| z1 only sets a scale: FP32).
#include <math.h>

#include <algorithm>
#include <vector>

#include "iter_ctx.cuh"
#include "lgk_impl.hpp"

namespace lgk {

constexpr int kChkCols = 16;     // columns per tile of the check products
constexpr int kChkBatch = 64;    // columns per pass (device temporaries)

// Element (i, p) of the iterations' A, in FP64: hi + lo (two BF16 terms),
// hi (one term), or the FP32 copy.
template <int NA>
__device__ inline double a_at(const void* A, size_t plane, size_t e) {
    if (NA == 0) return (double)static_cast<const float*>(A)[e];
    const __nv_bfloat16* h = static_cast<const __nv_bfloat16*>(A);
    double v = (double)__bfloat162float(h[e]);
    if (NA == 2) v += (double)__bfloat162float(h[plane + e]);
    return v;
}

// Z[c][p] = clip(q1[j][p], 0, u), Lam[c][i] = rho_j max(q2[j][i] - b, 0) for
// the listed columns j = cols[c], with the iteration's own (FP32) u, b and
// rho: the plan exactly as the library reports it.
__global__ void k_chk_prep(IterCtx cx, const int* __restrict__ cols, double* Z, double* Lam) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y, j = cols[c];
    if (e < cx.n_pad) {
        const int sl = cx.col_slot[e];
        const float u = u_at(cx, e, sl, j);
        Z[(size_t)c * cx.n_pad + e] = (double)fminf(fmaxf(cx.q1[(size_t)j * cx.n_pad + e], 0.f), u);
    }
    if (e < cx.m_pad) {
        double l = 0.0;
        if (e < cx.m) {
            const double q = cx.q2[(size_t)j * cx.m_pad + e];
            l = (double)cx.rho[j] * fmax(q - (double)b_of(e, j, cx.n_beams, cx.m, cx.Dr, cx.wbot), 0.0);
        }
        Lam[(size_t)c * cx.m_pad + e] = l;
    }
}

// AZ[c][i] = sum_p A[i][p] Z[c][p] (FP64), AZabs[c][i] = sum_p |A[i][p]| Z[c][p]
// (FP32).  Tile: 64 rows x 16 columns, k in steps of 32; thread (row, group of
// four columns).  Grid (m_pad / 64, ceil(nc / 16)), 256 threads.
template <int NA>
__global__ void __launch_bounds__(256) k_chk_az(const void* A, int m_pad, int n_pad, const double* Z, int nc,
                                                double* AZ, float* AZabs) {
    __shared__ double As[32][65];
    __shared__ double Zs[kChkCols][33];
    const int row0 = blockIdx.x * 64, c0 = blockIdx.y * kChkCols;
    const int r = threadIdx.x & 63, cg = threadIdx.x >> 6;
    const size_t plane = (size_t)m_pad * n_pad;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    float accab[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < n_pad; k0 += 32) {
        for (int e = threadIdx.x; e < 64 * 32; e += 256) {
            const int rr = e >> 5, kk = e & 31;
            As[kk][rr] = a_at<NA>(A, plane, (size_t)(row0 + rr) * n_pad + k0 + kk);
        }
        for (int e = threadIdx.x; e < kChkCols * 32; e += 256) {
            const int cc = e >> 5, kk = e & 31;
            Zs[cc][kk] = c0 + cc < nc ? Z[(size_t)(c0 + cc) * n_pad + k0 + kk] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const double a = As[kk][r];
            const float fa = fabsf((float)a);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const double z = Zs[cg * 4 + cc][kk];
                acc[cc] = fma(a, z, acc[cc]);
                accab[cc] = fmaf(fa, (float)z, accab[cc]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        const int c = c0 + cg * 4 + cc;
        if (c < nc) {
            AZ[(size_t)c * m_pad + row0 + r] = acc[cc];
            AZabs[(size_t)c * m_pad + row0 + r] = accab[cc];
        }
    }
}

// ATL[c][p] = sum_i A[i][p] Lam[c][i] (FP64).  Tile: 64 columns of A x 16
// plan columns, i in steps of 32.  Grid (n_pad / 64, ceil(nc / 16)), 256 threads.
template <int NA>
__global__ void __launch_bounds__(256) k_chk_atl(const void* A, int m_pad, int n_pad, const double* Lam, int nc,
                                                 double* ATL) {
    __shared__ double As[32][65];
    __shared__ double Ls[kChkCols][33];
    const int p0 = blockIdx.x * 64, c0 = blockIdx.y * kChkCols;
    const int p = threadIdx.x & 63, cg = threadIdx.x >> 6;
    const size_t plane = (size_t)m_pad * n_pad;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i0 = 0; i0 < m_pad; i0 += 32) {
        for (int e = threadIdx.x; e < 32 * 64; e += 256) {
            const int ii = e >> 6, pp = e & 63;
            As[ii][pp] = a_at<NA>(A, plane, (size_t)(i0 + ii) * n_pad + p0 + pp);
        }
        for (int e = threadIdx.x; e < kChkCols * 32; e += 256) {
            const int cc = e >> 5, ii = e & 31;
            Ls[cc][ii] = c0 + cc < nc ? Lam[(size_t)(c0 + cc) * m_pad + i0 + ii] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int ii = 0; ii < 32; ++ii) {
            const double a = As[ii][p];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) acc[cc] = fma(a, Ls[cg * 4 + cc][ii], acc[cc]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        const int c = c0 + cg * 4 + cc;
        if (c < nc) ATL[(size_t)c * n_pad + p0 + p] = acc[cc];
    }
}

// Block-wide sum / max over 256 threads in a fixed order (deterministic).
__device__ inline double blk_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double s = sh[0];
    __syncthreads();
    return s;
}

__device__ inline double blk_max(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    const double s = sh[0];
    __syncthreads();
    return s;
}

// One block per listed column: the check's quantities (see the file header)
// into out[c][LGK_CHECK_COUNT].  u64 [nc][n_slot] and wb64 [nc] hold the
// column's exact bounds and BOT weight (FP64).
__global__ void __launch_bounds__(256) k_chk_reduce(IterCtx cx, const int* __restrict__ cols,
                                                    const double* Z, const double* Lam, const double* AZ,
                                                    const float* AZabs, const double* ATL,
                                                    const double* __restrict__ u64,
                                                    const double* __restrict__ wb64, double* out) {
    __shared__ double sh[256];
    const int c = blockIdx.x, j = cols[c];
    double r2 = 0.0, s2 = 0.0, bl = 0.0, lmax = 0.0;
    for (int i = threadIdx.x; i < cx.m; i += 256) {
        const double b = i >= cx.n_beams ? wb64[c] * cx.Dr[i] : 0.0;
        const double v = fmax(AZ[(size_t)c * cx.m_pad + i] - b, 0.0);
        const double s = (double)AZabs[(size_t)c * cx.m_pad + i];
        const double l = Lam[(size_t)c * cx.m_pad + i];
        r2 += v * v;
        s2 += s * s;
        bl += b * l;
        lmax = fmax(lmax, l);
    }
    double obj = 0.0, hinge = 0.0, hard = 0.0, bound = 0.0;
    for (int p = threadIdx.x; p < cx.n; p += 256) {
        const int sl = cx.col_slot[p];
        const double cp = (double)cx.c_slot[sl];
        const double z = Z[(size_t)c * cx.n_pad + p];
        double u = u64[(size_t)c * cx.n_slot + sl];
        if (cx.mask && !((cx.mask[(size_t)p * cx.mask_words + (j >> 5)] >> (j & 31)) & 1u)) u = 0.0;
        const double neg = fmax(-(cp + ATL[(size_t)c * cx.n_pad + p]), 0.0);
        obj += cp * z;
        if (isinf(u)) {
            hard = fmax(hard, neg);
        } else {
            hinge += u * neg;
            bound = fmax(bound, z - u);
        }
    }
    r2 = blk_sum(r2, sh);
    s2 = blk_sum(s2, sh);
    bl = blk_sum(bl, sh);
    obj = blk_sum(obj, sh);
    hinge = blk_sum(hinge, sh);
    lmax = blk_max(lmax, sh);
    hard = blk_max(hard, sh);
    bound = blk_max(bound, sh);
    if (threadIdx.x == 0) {
        double* o = out + (size_t)c * LGK_CHECK_COUNT;
        const double plan = bl + hinge;
        o[LGK_CHECK_OBJ] = obj;
        o[LGK_CHECK_PLAN] = plan;
        o[LGK_CHECK_GAP] = (obj + plan) / fmax(1.0, fabs(obj));
        o[LGK_CHECK_INFEAS] = sqrt(r2) / fmax(sqrt(s2), 1e-300);
        o[LGK_CHECK_INFEAS_ABS] = sqrt(r2);
        o[LGK_CHECK_HARD] = hard / fmax(lmax, 1e-300);
        o[LGK_CHECK_BOUND] = bound;
    }
}

// Host: the check for the listed columns (host indices), out [nc][LGK_CHECK_COUNT]
// (host).  Runs on the case's stream in batches of kChkBatch columns, with
// device temporaries kept in r.chk for later calls.
int run_check(ResultData& r, const int* cols, int nc, double* out) {
    CaseData& cs = *r.cs;
    cudaStream_t st = cs.stream;
    if (nc <= 0) return LGK_OK;
    const int S = cs.n_slot;
    const size_t np = cs.n_pad, mp = cs.m_pad, B = kChkBatch;
    int rc;
    if (!r.chk.p) {
        // Z, ATL [B][n_pad] double; Lam, AZ [B][m_pad] double; AZabs [B][m_pad]
        // float; cols [B] int; u64 [B][S], wb64 [B], out [B][COUNT] double
        const size_t bytes = B * (2 * np + 2 * mp) * 8 + B * mp * 4 + B * 4 + B * (S + 1 + LGK_CHECK_COUNT) * 8;
        if ((rc = r.chk.alloc(round_up(bytes, 256) + 1024))) return rc;
    }
    char* base = static_cast<char*>(r.chk.p);
    auto take = [&](size_t n) {
        char* p = base;
        base += round_up(n, 256);
        return p;
    };
    double* Z = reinterpret_cast<double*>(take(B * np * 8));
    double* ATL = reinterpret_cast<double*>(take(B * np * 8));
    double* Lam = reinterpret_cast<double*>(take(B * mp * 8));
    double* AZ = reinterpret_cast<double*>(take(B * mp * 8));
    float* AZabs = reinterpret_cast<float*>(take(B * mp * 4));
    int* cols_d = reinterpret_cast<int*>(take(B * 4));
    double* u_d = reinterpret_cast<double*>(take(B * S * 8));
    double* wb_d = reinterpret_cast<double*>(take(B * 8));
    double* out_d = reinterpret_cast<double*>(take(B * LGK_CHECK_COUNT * 8));

    IterCtx cx = make_ctx_public(r);
    const void* A = cs.na ? cs.Ahat.p : cs.A32.p;
    std::vector<double> u_h(B * S), wb_h(B);
    for (int c0 = 0; c0 < nc; c0 += (int)B) {
        const int k = std::min((int)B, nc - c0);
        for (int c = 0; c < k; ++c) {
            const int j = cols[c0 + c];
            std::copy(&r.u64[(size_t)j * S], &r.u64[(size_t)j * S] + S, &u_h[(size_t)c * S]);
            wb_h[c] = r.wb64[j];
        }
        LGK_CUDA_TRY(cudaMemcpyAsync(cols_d, cols + c0, (size_t)k * 4, cudaMemcpyHostToDevice, st));
        LGK_CUDA_TRY(cudaMemcpyAsync(u_d, u_h.data(), (size_t)k * S * 8, cudaMemcpyHostToDevice, st));
        LGK_CUDA_TRY(cudaMemcpyAsync(wb_d, wb_h.data(), (size_t)k * 8, cudaMemcpyHostToDevice, st));
        const int ne = (int)std::max(np, mp);
        k_chk_prep<<<dim3((ne + 255) / 256, k), 256, 0, st>>>(cx, cols_d, Z, Lam);
        LGK_LAUNCH_CHECK();
        const dim3 gz((unsigned)(mp / 64), (k + kChkCols - 1) / kChkCols);
        const dim3 gl((unsigned)(np / 64), (k + kChkCols - 1) / kChkCols);
        if (cs.na == 2) {
            k_chk_az<2><<<gz, 256, 0, st>>>(A, (int)mp, (int)np, Z, k, AZ, AZabs);
            LGK_LAUNCH_CHECK();
            k_chk_atl<2><<<gl, 256, 0, st>>>(A, (int)mp, (int)np, Lam, k, ATL);
        } else if (cs.na == 1) {
            k_chk_az<1><<<gz, 256, 0, st>>>(A, (int)mp, (int)np, Z, k, AZ, AZabs);
            LGK_LAUNCH_CHECK();
            k_chk_atl<1><<<gl, 256, 0, st>>>(A, (int)mp, (int)np, Lam, k, ATL);
        } else {
            k_chk_az<0><<<gz, 256, 0, st>>>(A, (int)mp, (int)np, Z, k, AZ, AZabs);
            LGK_LAUNCH_CHECK();
            k_chk_atl<0><<<gl, 256, 0, st>>>(A, (int)mp, (int)np, Lam, k, ATL);
        }
        LGK_LAUNCH_CHECK();
        k_chk_reduce<<<k, 256, 0, st>>>(cx, cols_d, Z, Lam, AZ, AZabs, ATL, u_d, wb_d, out_d);
        LGK_LAUNCH_CHECK();
        LGK_CUDA_TRY(cudaMemcpyAsync(out + (size_t)c0 * LGK_CHECK_COUNT, out_d,
                                     (size_t)k * LGK_CHECK_COUNT * 8, cudaMemcpyDeviceToHost, st));
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return LGK_OK;
}

}  // namespace lgk
