// Iteration context shared by the element-wise kernels and the fused
// tensor-core epilogue: pointers and sizes of one solve, passed by value.
#pragma once

#include "lgk_common.cuh"

namespace lgk {

struct IterCtx {
    int Kp, m, m_pad, n_pad, n_beams, n_slot, check_every, max_iter;
    float tol;
    const uint8_t* col_slot;
    const float* utab;      // [Kp][n_slot]
    const uint32_t* mask;   // [n_pad][mask_words] point selection per column, or NULL (all)
    const float* c1;        // lo_refresh: [Kp][m_pad] lo R1 of the last full iteration, or NULL
    const float* c2;        // lo_refresh: [Kp][n_pad] lo^T v of the last full iteration, or NULL
    int mask_words;
    const float* c_slot;    // [n_slot] (stored after utab)
    const float* rho;       // colp[0]
    const float* inv_rho;   // colp[1]
    const float* wbot;      // colp[2]
    const float* refine_on; // colp[3]: 1 where the column's solve is refined (solve refinement)
    const double* Dr;
    float* q1;
    float* q2;
    int* active;            // [2][Kp]: active, converged
    int* iters;
    Control* ctrl;
    double* resid;          // [blocks][Kp][5]
    double* stats;          // [3][Kp]
    int n_resid_n, n_resid_m;
    double eps_abs;
    int n, m_rows;
};

// Upper bound u of point p (slot sl) in column j: the slot's bound, or 0 where
// the column's point selection leaves p out (Sec. 2.C, second pass).
__device__ inline float u_at(const IterCtx& cx, int p, int sl, int j) {
    float u = cx.utab[j * cx.n_slot + sl];
    if (cx.mask && !((cx.mask[(size_t)p * cx.mask_words + (j >> 5)] >> (j & 31)) & 1u)) u = 0.f;
    return u;
}

__device__ inline bool is_check_iter(const Control* c, int check_every, float tol) {
    int it = c->iter + 1;
    return (tol > 0.f && it % check_every == 0) || it >= c->max_iter;
}

// Stop test of column j after iteration `it` (Boyd et al. Sec. 3.3 on the
// residual partials of the n- and m-blocks, summed in a fixed order), run by
// all threads of the calling block (blockDim.x a multiple of 32, at most 32
// warps); red: 5 x (blockDim.x / 32) doubles of shared memory.  Records the
// column's iteration count and clears its active flag when it stops.
__device__ inline void finalize_column(const IterCtx& cx, int j, int it, bool err, double* red) {
    const bool check = (cx.tol > 0.f && it % cx.check_every == 0) || it >= cx.ctrl->max_iter;
    const bool test = cx.tol > 0.f && it % cx.check_every == 0;
    const int nw = blockDim.x >> 5;
    if (err) {
        if (threadIdx.x == 0) cx.active[j] = 0;
    } else if (cx.active[j]) {
        bool stop = it >= cx.ctrl->max_iter;
        if (check) {
            const int nb = cx.n_resid_n + cx.n_resid_m;
            double s5[5] = {0, 0, 0, 0, 0};
            for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
                for (int k = 0; k < 5; ++k) s5[k] += cx.resid[((size_t)b * cx.Kp + j) * 5 + k];
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                double v = s5[k];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) red[k * nw + w] = v;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double t5[5];
                for (int k = 0; k < 5; ++k) {
                    t5[k] = 0.0;
                    for (int q = 0; q < nw; ++q) t5[k] += red[k * nw + q];
                }
                const double sq = sqrt((double)(cx.n + cx.m_rows));
                const double rho = cx.rho[j];
                const double rn = sqrt(t5[0]), xn = sqrt(t5[1]), zn = sqrt(t5[2]);
                const double sn = rho * sqrt(t5[3]), yn = rho * sqrt(t5[4]);
                const double xz = fmax(xn, zn);
                cx.stats[j] = rn / fmax(xz, 1e-300);
                cx.stats[cx.Kp + j] = sn / fmax(yn, 1e-300);
                if (test && rn <= cx.eps_abs * sq + cx.tol * xz && sn <= cx.eps_abs * sq + cx.tol * yn) {
                    stop = true;
                    cx.active[cx.Kp + j] = 1;   // converged
                }
            }
        }
        if (threadIdx.x == 0) {
            cx.iters[j] = it;
            if (stop) cx.active[j] = 0;
        }
    }
}

// After every column's finalize_column (and a fence): count the active
// columns and advance the iteration counter (one block; cnt: a shared int).
__device__ inline void finalize_count(const IterCtx& cx, int it, int* cnt) {
    if (threadIdx.x == 0) *cnt = 0;
    __syncthreads();
    int mine = 0;
    for (int k = threadIdx.x; k < cx.Kp; k += blockDim.x) mine += ((volatile int*)cx.active)[k] != 0;
    atomicAdd(cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        Control* c = cx.ctrl;
        c->n_active = *cnt;
        c->iter = it;
        c->ticket = 0;
        __threadfence();
    }
}

__device__ inline float b_of(int i, int j, int n_beams, int m, const double* Dr, const float* wbot) {
    return (i >= n_beams && i < m) ? (float)(wbot[j] * Dr[i]) : 0.0f;
}

__device__ inline void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Column update of the n-block (q1) for one element, shared by both
// precisions: z = P1(q) = clip(q, 0, u), y = q - z;
//   q1' = P1(q1) - c/rho - w,  R1' = 2 P1(q1') - q1' - c/rho,
// and the residual terms r = y' - y, x = q1' - y, z', s = z' - z, y'.
struct Q1Update {
    float qn, r1, res[5];
};

__device__ inline Q1Update q1_update(float qo, float w, float u, float cr) {
    Q1Update o;
    float zo = fminf(fmaxf(qo, 0.f), u), yo = qo - zo;
    o.qn = zo - cr - w;
    float zn = fminf(fmaxf(o.qn, 0.f), u), yn = o.qn - zn;
    o.r1 = 2.f * zn - o.qn - cr;
    float r = yn - yo, x = o.qn - yo, s = zn - zo;
    o.res[0] = r * r; o.res[1] = x * x; o.res[2] = zn * zn; o.res[3] = s * s; o.res[4] = yn * yn;
    return o;
}

}  // namespace lgk
