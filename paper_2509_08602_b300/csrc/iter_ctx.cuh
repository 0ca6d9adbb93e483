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
