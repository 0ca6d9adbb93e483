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
//   infeas    ||(A z1 - b)_+||_2 / ||b||_2
//   infeas_abs ||(A z1 - b)_+||_2
//   hard      max over u = inf columns of (-(c + A^T lam))_+ / max lam
//             (organ limits and the BOT coupling, Appendix A)
//   bound     max over finite-u columns of (z1 - u)_+ (the iterations clip
//             to FP32 bounds)
//   primal    ||(A z1 - b)_+||_2 / ((1 + ||A||_2) ||z||_2), z = (z1, z2),
//             z2 = min(q2, b): a column that stopped with relative primal
//             residual r <= tol max(||x||, ||z||) has A z1 - b <= A (z1 - x1)
//             + (x2 - z2) + (A x1 - x2), so this is at most about tol when
//             the x-step's solve was accurate (A x1 - x2 = rhs - S v small);
//             a solve error shows up here and nowhere else
// A z1 and A^T lam: with A in two BF16 terms (the default form) on the tensor
// cores from exact splits -- z1 (FP32) is exactly three BF16 terms, lam is
// rounded to three (2^-24) -- with 5 exact BF16 products, FP32 sums over
// stream-K segments of one 64-column k block and FP64 sums across segments;
// otherwise (or with check_fp64) FP64 dot products on the CUDA cores.
// Everything after the two products is FP64.
#include <math.h>

#include <algorithm>
#include <vector>

#include "iter_ctx.cuh"
#include "lgk_impl.hpp"
#include "tc_ptx.cuh"

namespace lgk {

constexpr int kChkCols = 8;      // columns per tile of the check products (2 per thread)
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

// Per-column inputs of one check batch: the state columns (q1 [.][n_pad], q2
// [.][m_pad] FP32, column src[c]) and the FP32 tables the iteration used
// for them (u per slot, rho, w_BOT), plus the exact FP64 tables of the LP.
struct ChkCols {
    const float* q1;
    const float* q2;
    const int* src;        // [nc] state column
    const int* mcol;       // [nc] point-selection column, or null (no selection)
    const float* uf;       // [nc][n_slot]
    const float* rhof;     // [nc]
    const float* wbf;      // [nc]
    const double* u64;     // [nc][n_slot]
    const double* wb64;    // [nc]
};

__device__ inline float chk_b(const IterCtx& cx, int i, float wb) {
    return (i >= cx.n_beams && i < cx.m) ? (float)(wb * cx.Dr[i]) : 0.0f;   // as the iteration's b
}

__device__ inline bool chk_selected(const IterCtx& cx, const ChkCols& k, int c, int p) {
    if (!cx.mask || !k.mcol) return true;
    const int j = k.mcol[c];
    return (cx.mask[(size_t)p * cx.mask_words + (j >> 5)] >> (j & 31)) & 1u;
}

// Z[c][p] = clip(q1, 0, u), Lam[c][i] = rho max(q2 - b, 0): the plan exactly
// as the library reports it (FP32 u, b, rho of the iteration).
__global__ void k_chk_prep(IterCtx cx, ChkCols k, double* Z, double* Lam) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y, j = k.src[c];
    if (e < cx.n_pad) {
        const int sl = cx.col_slot[e];
        const float u = chk_selected(cx, k, c, e) ? k.uf[(size_t)c * cx.n_slot + sl] : 0.0f;
        Z[(size_t)c * cx.n_pad + e] = (double)fminf(fmaxf(k.q1[(size_t)j * cx.n_pad + e], 0.f), u);
    }
    if (e < cx.m_pad) {
        double l = 0.0;
        if (e < cx.m) {
            const double q = k.q2[(size_t)j * cx.m_pad + e];
            l = (double)k.rhof[c] * fmax(q - (double)chk_b(cx, e, k.wbf[c]), 0.0);
        }
        Lam[(size_t)c * cx.m_pad + e] = l;
    }
}

// AZ[c][i] = sum_p A[i][p] Z[c][p] (FP64).  Tile: 64 rows x 8 columns, k in
// steps of 32; thread (row, two columns).  Grid (m_pad / 64, ceil(nc / 8)),
// 256 threads.
template <int NA>
__global__ void __launch_bounds__(256) k_chk_az(const void* A, int m_pad, int n_pad, const double* Z, int nc,
                                                double* AZ) {
    __shared__ double As[32][65];
    __shared__ double Zs[kChkCols][33];
    const int row0 = blockIdx.x * 64, c0 = blockIdx.y * kChkCols;
    const int r = threadIdx.x & 63, cg = threadIdx.x >> 6;
    const size_t plane = (size_t)m_pad * n_pad;
    constexpr int CT = kChkCols / 4;      // columns per thread
    double acc[CT] = {};
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
#pragma unroll
            for (int cc = 0; cc < CT; ++cc) acc[cc] = fma(a, Zs[cg * CT + cc][kk], acc[cc]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) {
        const int c = c0 + cg * CT + cc;
        if (c < nc) AZ[(size_t)c * m_pad + row0 + r] = acc[cc];
    }
}

// ATL[c][p] = sum_i A[i][p] Lam[c][i] (FP64).  Tile: 64 columns of A x 8
// plan columns, i in steps of 32.  Grid (n_pad / 64, ceil(nc / 8)), 256 threads.
template <int NA>
__global__ void __launch_bounds__(256) k_chk_atl(const void* A, int m_pad, int n_pad, const double* Lam, int nc,
                                                 double* ATL) {
    __shared__ double As[32][65];
    __shared__ double Ls[kChkCols][33];
    const int p0 = blockIdx.x * 64, c0 = blockIdx.y * kChkCols;
    const int p = threadIdx.x & 63, cg = threadIdx.x >> 6;
    const size_t plane = (size_t)m_pad * n_pad;
    constexpr int CT = kChkCols / 4;
    double acc[CT] = {};
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
            for (int cc = 0; cc < CT; ++cc) acc[cc] = fma(a, Ls[cg * CT + cc][ii], acc[cc]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) {
        const int c = c0 + cg * CT + cc;
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
// into out[c][LGK_CHECK_COUNT].
__global__ void __launch_bounds__(256) k_chk_reduce(IterCtx cx, ChkCols k, const double* Z, const double* Lam,
                                                    const double* AZ, const double* ATL, double a_norm,
                                                    double* out) {
    __shared__ double sh[256];
    const int c = blockIdx.x, j = k.src[c];
    double r2 = 0.0, s2 = 0.0, bl = 0.0, lmax = 0.0, z2 = 0.0;
    for (int i = threadIdx.x; i < cx.m; i += 256) {
        const double b = i >= cx.n_beams ? k.wb64[c] * cx.Dr[i] : 0.0;
        const double v = fmax(AZ[(size_t)c * cx.m_pad + i] - b, 0.0);
        const double s = b;
        const double l = Lam[(size_t)c * cx.m_pad + i];
        const double zz = (double)fminf(k.q2[(size_t)j * cx.m_pad + i], chk_b(cx, i, k.wbf[c]));
        r2 += v * v;
        s2 += s * s;
        bl += b * l;
        lmax = fmax(lmax, l);
        z2 += zz * zz;
    }
    double obj = 0.0, hinge = 0.0, hard = 0.0, bound = 0.0, z1 = 0.0;
    for (int p = threadIdx.x; p < cx.n; p += 256) {
        const int sl = cx.col_slot[p];
        const double cp = (double)cx.c_slot[sl];
        const double z = Z[(size_t)c * cx.n_pad + p];
        const double u = chk_selected(cx, k, c, p) ? k.u64[(size_t)c * cx.n_slot + sl] : 0.0;
        const double neg = fmax(-(cp + ATL[(size_t)c * cx.n_pad + p]), 0.0);
        obj += cp * z;
        z1 += z * z;
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
    z1 = blk_sum(z1, sh);
    z2 = blk_sum(z2, sh);
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
        o[LGK_CHECK_PRIMAL] = sqrt(r2) / fmax((1.0 + a_norm) * sqrt(z1 + z2), 1e-300);
    }
}

// Split operands of the tensor-core products: Z3 / L3 [3][kCheckCols][n_pad
// resp. m_pad] BF16 (hi, mid, lo) of z1 and lam (columns past nc are zero).
__global__ void k_chk_split(const double* Z, const double* Lam, int nc, int n_pad, int m_pad,
                            __nv_bfloat16* z3, __nv_bfloat16* l3) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
    auto split = [](double x, __nv_bfloat16* d, size_t plane) {
        const __nv_bfloat16 h = bf16_from_double(x);
        const double r1 = x - (double)__bfloat162float(h);
        const __nv_bfloat16 m = bf16_from_double(r1);
        d[0] = h;
        d[plane] = m;
        d[2 * plane] = bf16_from_double(r1 - (double)__bfloat162float(m));
    };
    if (e < n_pad)
        split(c < nc ? Z[(size_t)c * n_pad + e] : 0.0, z3 + (size_t)c * n_pad + e, (size_t)kCheckCols * n_pad);
    if (e < m_pad)
        split(c < nc ? Lam[(size_t)c * m_pad + e] : 0.0, l3 + (size_t)c * m_pad + e, (size_t)kCheckCols * m_pad);
}

// out[c][i] = sum of the product's stream-K segment partials of row i,
// column c, in k order, in FP64 (one column tile of kCheckCols columns).
// Grid (rows_pad / 128, kCheckCols), 128 threads.
__global__ void k_chk_sum(const float* __restrict__ part, const int* __restrict__ tile_begin, int rows_pad,
                          double* out) {
    const int t = blockIdx.x, c = blockIdx.y, r = threadIdx.x;
    const int b = tile_begin[t], e = tile_begin[t + 1];
    double s = 0.0;
    for (int k = b; k < e; ++k) s += (double)__ldcg(part + ((size_t)k * kCheckCols + c) * 128 + r);
    out[(size_t)c * rows_pad + t * 128 + r] = s;
}

static int check_tc_setup(CaseData& cs) {
    if (cs.chk_tc) return LGK_OK;
    std::unique_ptr<CheckTC> k(new CheckTC);
    const int mp = cs.m_pad, np = cs.n_pad;
    int rc;
    if ((rc = build_plan(k->az, mp / 128, 1, np / 64, kCheckCols, false, 1, 1))) return rc;
    if ((rc = build_plan(k->atl, np / 128, 1, mp / 64, kCheckCols, false, 1, 1))) return rc;
    if ((rc = k->part.alloc((size_t)std::max(k->az.nseg, k->atl.nseg) * kCheckCols * 128 * 4))) return rc;
    if ((rc = k->z3.alloc((size_t)3 * kCheckCols * np * 2)) || (rc = k->l3.alloc((size_t)3 * kCheckCols * mp * 2)))
        return rc;
    if ((rc = k->ctrl.alloc(sizeof(Control)))) return rc;
    const Control c0{1, 1, 1 << 30, 0, 0};       // work to do, no error
    LGK_CUDA_TRY(cudaMemcpy(k->ctrl.p, &c0, sizeof(c0), cudaMemcpyHostToDevice));
    if ((rc = make_tma_map(&k->mA_k, cs.Ahat.p, np, mp, 2, 128))) return rc;
    if ((rc = make_tma_map(&k->mA_mn, cs.Ahat.p, np, mp, 2, 64))) return rc;
    if ((rc = make_tma_map(&k->mZ, k->z3.p, np, kCheckCols, 3, kCheckCols))) return rc;
    if ((rc = make_tma_map(&k->mL, k->l3.p, mp, kCheckCols, 3, kCheckCols))) return rc;
    cs.chk_tc = std::move(k);
    return LGK_OK;
}

// Host: the check of nc state columns (q1 [.][n_pad], q2 [.][m_pad] on the
// device, column src[c]) with their FP32 tables (uf [nc][n_slot], rhof, wbf),
// exact tables (u64 [nc][n_slot], wb64) and point-selection columns (mcol, or
// null) -> out [nc][LGK_CHECK_COUNT] (host).  Runs on the case's stream in
// batches of kChkBatch columns, with device temporaries kept in r.chk.
int run_check_states(ResultData& r, const float* q1, const float* q2, int nc, const int* src, const int* mcol,
                     const float* uf, const float* rhof, const float* wbf, const double* u64,
                     const double* wb64, double* out) {
    CaseData& cs = *r.cs;
    cudaStream_t st = cs.stream;
    if (nc <= 0) return LGK_OK;
    const int S = cs.n_slot;
    const size_t np = cs.n_pad, mp = cs.m_pad, B = kChkBatch;
    int rc;
    // Z, ATL [B][n_pad] double; Lam, AZ [B][m_pad] double;
    // per column: src, mcol (int), uf (float S), rhof, wbf (float), u64 (double S), wb64 (double); out
    const size_t tab = round_up(B * 8, 256) + round_up(B * (S + 2) * 4, 256) + round_up(B * (S + 1) * 8, 256) +
                       round_up(B * LGK_CHECK_COUNT * 8, 256);
    const size_t bytes = B * (2 * np + 2 * mp) * 8 + tab;
    const bool tc = cs.na == 2 && !cs.prm.check_fp64;
    if (tc && (rc = check_tc_setup(cs))) return rc;
    if (r.chk.bytes < bytes && (rc = r.chk.alloc(bytes))) return rc;
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
    int* src_d = reinterpret_cast<int*>(take(B * 8));       // src [B], mcol [B]
    float* f_d = reinterpret_cast<float*>(take(B * (S + 2) * 4));
    double* d_d = reinterpret_cast<double*>(take(B * (S + 1) * 8));
    double* out_d = reinterpret_cast<double*>(take(B * LGK_CHECK_COUNT * 8));

    IterCtx cx = make_ctx_public(r);
    const void* A = cs.na ? cs.Ahat.p : cs.A32.p;
    std::vector<int> ih(2 * B);
    std::vector<float> fh(B * (S + 2));
    std::vector<double> dh(B * (S + 1));
    for (int c0 = 0; c0 < nc; c0 += (int)B) {
        const int k = std::min((int)B, nc - c0);
        for (int c = 0; c < k; ++c) {
            ih[c] = src[c0 + c];
            ih[B + c] = mcol ? mcol[c0 + c] : 0;
            std::copy(uf + (size_t)(c0 + c) * S, uf + (size_t)(c0 + c + 1) * S, &fh[(size_t)c * S]);
            fh[B * S + c] = rhof[c0 + c];
            fh[B * S + B + c] = wbf[c0 + c];
            std::copy(u64 + (size_t)(c0 + c) * S, u64 + (size_t)(c0 + c + 1) * S, &dh[(size_t)c * S]);
            dh[B * S + c] = wb64[c0 + c];
        }
        LGK_CUDA_TRY(cudaMemcpyAsync(src_d, ih.data(), ih.size() * 4, cudaMemcpyHostToDevice, st));
        LGK_CUDA_TRY(cudaMemcpyAsync(f_d, fh.data(), fh.size() * 4, cudaMemcpyHostToDevice, st));
        LGK_CUDA_TRY(cudaMemcpyAsync(d_d, dh.data(), dh.size() * 8, cudaMemcpyHostToDevice, st));
        ChkCols kc{q1, q2, src_d, mcol ? src_d + B : nullptr, f_d, f_d + B * S, f_d + B * S + B, d_d, d_d + B * S};
        const int ne = (int)std::max(np, mp);
        k_chk_prep<<<dim3((ne + 255) / 256, k), 256, 0, st>>>(cx, kc, Z, Lam);
        LGK_LAUNCH_CHECK();
        if (tc) {
            // passes of kCheckCols columns through the two tensor-core products
            CheckTC& t = *cs.chk_tc;
            IterCtx pc = cx;
            pc.ctrl = t.ctrl.as<Control>();
            for (int p0 = 0; p0 < k; p0 += kCheckCols) {
                const int kk = std::min(kCheckCols, k - p0);
                k_chk_split<<<dim3((ne + 255) / 256, kCheckCols), 256, 0, st>>>(
                    Z + (size_t)p0 * np, Lam + (size_t)p0 * mp, kk, (int)np, (int)mp, t.z3.as<__nv_bfloat16>(),
                    t.l3.as<__nv_bfloat16>());
                LGK_LAUNCH_CHECK();
                if ((rc = tc_check_product(cs, false, t.mA_k, t.mZ, t.az, pc, t.part.as<float>(), st))) return rc;
                k_chk_sum<<<dim3((unsigned)(mp / 128), kCheckCols), 128, 0, st>>>(t.part.as<float>(), t.az.tile_begin,
                                                                                 (int)mp, AZ + (size_t)p0 * mp);
                LGK_LAUNCH_CHECK();
                if ((rc = tc_check_product(cs, true, t.mA_mn, t.mL, t.atl, pc, t.part.as<float>(), st))) return rc;
                k_chk_sum<<<dim3((unsigned)(np / 128), kCheckCols), 128, 0, st>>>(t.part.as<float>(), t.atl.tile_begin,
                                                                                 (int)np, ATL + (size_t)p0 * np);
                LGK_LAUNCH_CHECK();
            }
        } else {
            const dim3 gz((unsigned)(mp / 64), (k + kChkCols - 1) / kChkCols);
            const dim3 gl((unsigned)(np / 64), (k + kChkCols - 1) / kChkCols);
            if (cs.na == 2) {
                k_chk_az<2><<<gz, 256, 0, st>>>(A, (int)mp, (int)np, Z, k, AZ);
                LGK_LAUNCH_CHECK();
                k_chk_atl<2><<<gl, 256, 0, st>>>(A, (int)mp, (int)np, Lam, k, ATL);
            } else if (cs.na == 1) {
                k_chk_az<1><<<gz, 256, 0, st>>>(A, (int)mp, (int)np, Z, k, AZ);
                LGK_LAUNCH_CHECK();
                k_chk_atl<1><<<gl, 256, 0, st>>>(A, (int)mp, (int)np, Lam, k, ATL);
            } else {
                k_chk_az<0><<<gz, 256, 0, st>>>(A, (int)mp, (int)np, Z, k, AZ);
                LGK_LAUNCH_CHECK();
                k_chk_atl<0><<<gl, 256, 0, st>>>(A, (int)mp, (int)np, Lam, k, ATL);
            }
            LGK_LAUNCH_CHECK();
        }
        k_chk_reduce<<<k, 256, 0, st>>>(cx, kc, Z, Lam, AZ, ATL, cs.a_norm, out_d);
        LGK_LAUNCH_CHECK();
        LGK_CUDA_TRY(cudaMemcpyAsync(out + (size_t)c0 * LGK_CHECK_COUNT, out_d,
                                     (size_t)k * LGK_CHECK_COUNT * 8, cudaMemcpyDeviceToHost, st));
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
        if (tc) {
            Control h{};
            LGK_CUDA_TRY(cudaMemcpy(&h, cs.chk_tc->ctrl.p, sizeof(h), cudaMemcpyDeviceToHost));
            if (h.err) {
                set_error("plan check: device error flag " + std::to_string(h.err));
                return LGK_ECUDA;
            }
        }
    }
    return LGK_OK;
}

// The check of live columns of a solve (their current state and tables).
int run_check(ResultData& r, const int* cols, int nc, double* out) {
    const int S = r.cs->n_slot, Kp = r.Kp;
    std::vector<float> uf((size_t)nc * S), rhof(nc), wbf(nc);
    std::vector<double> u64((size_t)nc * S), wb64(nc);
    for (int c = 0; c < nc; ++c) {
        const int j = cols[c];
        for (int s = 0; s < S; ++s) {
            u64[(size_t)c * S + s] = r.u64[(size_t)j * S + s];
            uf[(size_t)c * S + s] = (float)r.u64[(size_t)j * S + s];
        }
        rhof[c] = r.colp_h[j];
        wbf[c] = r.colp_h[2 * (size_t)Kp + j];
        wb64[c] = r.wb64[j];
    }
    return run_check_states(r, r.q1.as<float>(), r.q2.as<float>(), nc, cols, r.mask_words ? cols : nullptr,
                            uf.data(), rhof.data(), wbf.data(), u64.data(), wb64.data(), out);
}

}  // namespace lgk
