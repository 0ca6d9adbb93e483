// One ADMM solve over K weightings (Sec. 2.B), in the q-form used on the
// device.  With q1 = x1 + y1_prev and q2 = x2 + y2_prev, z = P(q) and
// y = q - P(q), and one iteration of Eq. admm (x-step in the closed form of
// Eq. partial_elimination) reads
//     rhs = A (2 P1(q1) - q1 - c/rho) + q2 - 2 P2(q2)
//     v   = S^{-1} rhs
//     q1' = P1(q1) - c/rho - A^T v,      q2' = v + P2(q2)
// with P1 = clip to [0, u] and P2 = min(., b).  The state is one n x K and one
// m x K matrix; weightings are the K columns.
//
// Kernel sequence of one iteration (both precisions):
//   GEMM1      part = A . R1
//   reduce     rhs  = part + q2 - 2 P2(q2)
//   solve      part = S^{-1} . rhs
//   reduce     q2'  = part + P2(q2), residual partials of the m-block
//   GEMM2      part = A^T . V
//   q1 update  q1'  = P1(q1) - c/rho - part, R1' for the next GEMM1, residual
//              partials of the n-block
//   finalize   per-column stop test (Boyd et al. Sec. 3.3), freeze
// The BF16 forms' GEMMs leave stream-K segment partials that the next kernel
// sums per element in k order; the FP32 form's cuBLAS GEMMs leave a plain
// matrix.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <chrono>
#include <thread>
#include <vector>

#include "lgk_impl.hpp"
#include "iter_ctx.cuh"

namespace lgk {

ResultData::~ResultData() {
    if (worker.joinable()) {      // an asynchronous solve still running: stop it at its next replay
        cancel = true;
        worker.join();
    }
    if (cs && cs->stream) cudaStreamSynchronize(cs->stream);
    if (graph) cudaGraphExecDestroy(graph);
    for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
}

// Event before kernel k of captured iteration `it` (profile mode).
static void prof_mark(ResultData& r, int it, int k) {
    // External: captured as an event-record node of the graph (a plain record
    // inside a capture only expresses a dependency)
    if (!r.prof_ev.empty())
        cudaEventRecordWithFlags(r.prof_ev[(size_t)it * (r.prof_class.size() + 1) + k], r.cs->stream,
                                 cudaEventRecordExternal);
}

// ---------------------------------------------------------------- helpers

// Where one GEMM's output lives: a plain [Kp][rows_pad] matrix (tile_begin
// null), or stream-K segment slots [slot][n_tile][128] summed in k order.
struct SumSrc {
    const float* part;
    const int* tile_begin;
    const int* tile_slots;
    int rows_pad, row_tiles, n_tile;
    int mt;                 // 128-row sub-tiles per tile: slots are [slot][mt][n_tile][128]
};

// Sum of the GEMM output at (i, j): the plain matrix, or the tile's slots.
// Slots of a tile are contiguous ([tile_begin[t], tile_begin[t + 1])), so the
// loads of the different slots are independent of each other.
__device__ inline float gemm_out(const SumSrc& s, int i, int j) {
    if (!s.tile_begin) return s.part[(size_t)j * s.rows_pad + i];
    const int ct = j / s.n_tile, t = ct * s.row_tiles + (i >> 7) / s.mt, h = (i >> 7) % s.mt;
    const int b = __ldg(s.tile_begin + t), e = __ldg(s.tile_begin + t + 1);
    const float* p = s.part + (((size_t)b * s.mt + h) * s.n_tile + (j - ct * s.n_tile)) * 128 + (i & 127);
    const size_t stride = (size_t)s.mt * s.n_tile * 128;
    float acc = 0.f;
    int k = 0;
    for (; k + 4 <= e - b; k += 4) {
        const float a0 = __ldcg(p + k * stride), a1 = __ldcg(p + (k + 1) * stride);
        const float a2 = __ldcg(p + (k + 2) * stride), a3 = __ldcg(p + (k + 3) * stride);
        acc += a0;
        acc += a1;
        acc += a2;
        acc += a3;
    }
    for (; k < e - b; ++k) acc += __ldcg(p + k * stride);
    return acc;
}

// The same for rows i .. i+3 (i % 4 == 0, one 16-byte load per slot): the
// slots of a tile hold 128 consecutive rows per column, so four rows of one
// column are one aligned float4.
__device__ inline float4 gemm_out4(const SumSrc& s, int i, int j) {
    if (!s.tile_begin) return __ldcg(reinterpret_cast<const float4*>(s.part + (size_t)j * s.rows_pad + i));
    const int ct = j / s.n_tile, t = ct * s.row_tiles + (i >> 7) / s.mt, h = (i >> 7) % s.mt;
    const int b = __ldg(s.tile_begin + t), e = __ldg(s.tile_begin + t + 1);
    const float4* p = reinterpret_cast<const float4*>(
        s.part + (((size_t)b * s.mt + h) * s.n_tile + (j - ct * s.n_tile)) * 128 + (i & 127));
    const size_t stride = (size_t)s.mt * s.n_tile * 32;      // in float4
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int k = 0;
    for (; k + 4 <= e - b; k += 4) {
        const float4 a0 = __ldcg(p + k * stride), a1 = __ldcg(p + (k + 1) * stride);
        const float4 a2 = __ldcg(p + (k + 2) * stride), a3 = __ldcg(p + (k + 3) * stride);
        acc.x += a0.x; acc.y += a0.y; acc.z += a0.z; acc.w += a0.w;
        acc.x += a1.x; acc.y += a1.y; acc.z += a1.z; acc.w += a1.w;
        acc.x += a2.x; acc.y += a2.y; acc.z += a2.z; acc.w += a2.w;
        acc.x += a3.x; acc.y += a3.y; acc.z += a3.z; acc.w += a3.w;
    }
    for (; k < e - b; ++k) {
        const float4 a = __ldcg(p + k * stride);
        acc.x += a.x; acc.y += a.y; acc.z += a.z; acc.w += a.w;
    }
    return acc;
}

__device__ inline float f4(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

__device__ inline void block_sum5(float v[5], double* out) {
    __shared__ float red[5][8];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        float s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[k][w] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double s = 0.0;
            for (int i = 0; i < nw; ++i) s += (double)red[k][i];
            out[k] = s;
        }
    }
}

// R1 = 2 P1(q1) - q1 - c/rho for the first GEMM1 (q1 = 0 at the start).
template <bool BF16>
__global__ void k_init_r1(IterCtx cx, void* R1) {
    int p = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (p >= cx.n_pad) return;
    int sl = cx.col_slot[p];
    float u = u_at(cx, p, sl, j);
    float cr = cx.c_slot[sl] * cx.inv_rho[j];
    float q = cx.q1[(size_t)j * cx.n_pad + p];
    float z = fminf(fmaxf(q, 0.f), u);
    float r = 2.f * z - q - cr;
    size_t o = (size_t)j * cx.n_pad + p;
    if (BF16) {
        __nv_bfloat16 hi, lo;
        split_bf16(r, hi, lo);
        static_cast<__nv_bfloat16*>(R1)[o] = hi;
        static_cast<__nv_bfloat16*>(R1)[(size_t)cx.Kp * cx.n_pad + o] = lo;
    } else {
        static_cast<float*>(R1)[o] = r;
    }
}

// rhs = A R1 (+ the lagged lo R1) + q2 - 2 P2(q2), split into three BF16
// parts (the solve amplifies input rounding).  Four rows per thread; grid
// (m_pad / 256, Kp), 64 threads.
template <bool BF16>
__device__ __forceinline__ void reduce_rhs_body(const IterCtx& cx, const SumSrc& src, void* rhs, float* rhs32,
                                                int bx, int j) {
    if (cx.ctrl->n_active == 0 || cx.ctrl->err) return;
    const int i = bx * 256 + threadIdx.x * 4;
    const size_t o = (size_t)j * cx.m_pad + i;
    const float4 acc = gemm_out4(src, i, j);
    const float4 c1 = cx.c1 ? __ldcg(reinterpret_cast<const float4*>(cx.c1 + o)) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 q = *reinterpret_cast<const float4*>(cx.q2 + o);
    float r[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float p2 = fminf(f4(q, k), b_of(i + k, j, cx.n_beams, cx.m, cx.Dr, cx.wbot));
        r[k] = f4(acc, k) + f4(c1, k) + f4(q, k) - 2.f * p2;
    }
    if (BF16) {
        const size_t plane = (size_t)cx.Kp * cx.m_pad;
        __nv_bfloat16 hi[4], mid[4], lo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            hi[k] = __float2bfloat16_rn(r[k]);
            const float r1 = r[k] - __bfloat162float(hi[k]);
            mid[k] = __float2bfloat16_rn(r1);
            lo[k] = __float2bfloat16_rn(r1 - __bfloat162float(mid[k]));
        }
        __nv_bfloat16* d = static_cast<__nv_bfloat16*>(rhs) + o;
        *reinterpret_cast<uint2*>(d) = *reinterpret_cast<const uint2*>(hi);
        *reinterpret_cast<uint2*>(d + plane) = *reinterpret_cast<const uint2*>(mid);
        *reinterpret_cast<uint2*>(d + 2 * plane) = *reinterpret_cast<const uint2*>(lo);
        if (rhs32) *reinterpret_cast<float4*>(rhs32 + o) = make_float4(r[0], r[1], r[2], r[3]);
    } else {
        *reinterpret_cast<float4*>(static_cast<float*>(rhs) + o) = make_float4(r[0], r[1], r[2], r[3]);
    }
}

template <bool BF16>
__global__ void __launch_bounds__(64) k_reduce_rhs(IterCtx cx, SumSrc src, void* rhs, float* rhs32) {
    pdl_trigger();
    pdl_wait();
    reduce_rhs_body<BF16>(cx, src, rhs, rhs32, blockIdx.x, blockIdx.y);
}

__device__ inline void split3_store(const float v[4], __nv_bfloat16* d, size_t plane) {
    __nv_bfloat16 hi[4], mid[4], lo[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        hi[k] = __float2bfloat16_rn(v[k]);
        const float r1 = v[k] - __bfloat162float(hi[k]);
        mid[k] = __float2bfloat16_rn(r1);
        lo[k] = __float2bfloat16_rn(r1 - __bfloat162float(mid[k]));
    }
    *reinterpret_cast<uint2*>(d) = *reinterpret_cast<const uint2*>(hi);
    *reinterpret_cast<uint2*>(d + plane) = *reinterpret_cast<const uint2*>(mid);
    *reinterpret_cast<uint2*>(d + 2 * plane) = *reinterpret_cast<const uint2*>(lo);
}

// Refinement of the solve (lgk_params.solve_refine): e = rhs - S v, with
// rhs kept in FP32 by k_reduce_rhs and S v summed from the S . V3 product's
// stream-K slots; e goes into the solve's input planes (three BF16 terms) for
// the next product with S^{-1}.  A column whose refinement is off
// (refine_on = 0: refine_after, the column is younger than the limit) gets
// e = 0, so its correction S^{-1} e is exactly zero and its v is bitwise the
// unrefined solve's.  Grid (m_pad / 256, Kp), 64 threads.
__device__ __forceinline__ void reduce_err_body(const IterCtx& cx, const SumSrc& src, const float* rhs32,
                                                __nv_bfloat16* rhs, int bx, int j) {
    if (cx.ctrl->n_active == 0 || cx.ctrl->err) return;
    const int i = bx * 256 + threadIdx.x * 4;
    const size_t o = (size_t)j * cx.m_pad + i;
    const float4 sv = gemm_out4(src, i, j);
    const float4 b = *reinterpret_cast<const float4*>(rhs32 + o);
    float e[4] = {b.x - sv.x, b.y - sv.y, b.z - sv.z, b.w - sv.w};
    if (cx.refine_on[j] == 0.f) e[0] = e[1] = e[2] = e[3] = 0.f;
    split3_store(e, rhs + o, (size_t)cx.Kp * cx.m_pad);
}

__global__ void __launch_bounds__(64) k_reduce_err(IterCtx cx, SumSrc src, const float* __restrict__ rhs32,
                                                   __nv_bfloat16* rhs) {
    pdl_trigger();
    pdl_wait();
    reduce_err_body(cx, src, rhs32, rhs, blockIdx.x, blockIdx.y);
}

// v = S^{-1} rhs;  q2' = v + P2(q2);  residual partials of the m-block (one
// per 128-row tile and column: one warp per 128 rows, four rows per thread).
// Grid (m_pad / 256, Kp), 64 threads.
// MODE (solve refinement, lgk_params.solve_refine):
//   RS_PLAIN  v = S^{-1} rhs from the slots; the q2 step below
//   RS_FIRST  v0 = the slots: kept in FP32 (rv) and as three BF16 terms (V3)
//             for the refinement's S v0; no state update yet
//   RS_ACCUM  v = rv + the slots (a correction S^{-1} e), kept as RS_FIRST
//   RS_FINAL  v = rv + the slots; the q2 step below
enum { RS_PLAIN = 0, RS_FIRST = 1, RS_FINAL = 2, RS_ACCUM = 3 };

template <bool BF16, int MODE>
__device__ __forceinline__ void reduce_solve_body(const IterCtx& cx, const SumSrc& src, void* V, float* rv,
                                                  __nv_bfloat16* V3, int bx, int j) {
    if (cx.ctrl->n_active == 0 || cx.ctrl->err) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rt = bx * 2 + w, i = rt * 128 + lane * 4;
    const size_t o = (size_t)j * cx.m_pad + i;
    float4 v = gemm_out4(src, i, j);
    if (MODE == RS_ACCUM || MODE == RS_FINAL) {
        const float4 p = *reinterpret_cast<const float4*>(rv + o);
        v = make_float4(p.x + v.x, p.y + v.y, p.z + v.z, p.w + v.w);
    }
    if (MODE == RS_FIRST || MODE == RS_ACCUM) {
        *reinterpret_cast<float4*>(rv + o) = v;
        const float vv[4] = {v.x, v.y, v.z, v.w};
        split3_store(vv, V3 + o, (size_t)cx.Kp * cx.m_pad);
        return;
    }
    const bool check = is_check_iter(cx.ctrl, cx.check_every, cx.tol);
    const float4 qo = *reinterpret_cast<const float4*>(cx.q2 + o);
    float qn[4], res[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float bb = b_of(i + k, j, cx.n_beams, cx.m, cx.Dr, cx.wbot);
        const float zo = fminf(f4(qo, k), bb);
        qn[k] = f4(v, k) + zo;
        const float yo = f4(qo, k) - zo, zn = fminf(qn[k], bb), yn = qn[k] - zn;
        const float r = yn - yo, x = qn[k] - yo, sres = zn - zo;
        res[0] += r * r; res[1] += x * x; res[2] += zn * zn; res[3] += sres * sres; res[4] += yn * yn;
    }
    if (cx.active[j]) *reinterpret_cast<float4*>(cx.q2 + o) = make_float4(qn[0], qn[1], qn[2], qn[3]);
    if (BF16) {
        __nv_bfloat16 hi[4], lo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) split_bf16(f4(v, k), hi[k], lo[k]);
        __nv_bfloat16* d = static_cast<__nv_bfloat16*>(V) + o;
        *reinterpret_cast<uint2*>(d) = *reinterpret_cast<const uint2*>(hi);
        *reinterpret_cast<uint2*>(d + (size_t)cx.Kp * cx.m_pad) = *reinterpret_cast<const uint2*>(lo);
    } else {
        *reinterpret_cast<float4*>(static_cast<float*>(V) + o) = v;
    }
    if (check) {
#pragma unroll
        for (int k = 0; k < 5; ++k)
            for (int sh = 16; sh > 0; sh >>= 1) res[k] += __shfl_xor_sync(0xffffffffu, res[k], sh);
        if (lane == 0) {
            double* dst = cx.resid + ((size_t)(cx.n_resid_n + rt) * cx.Kp + j) * 5;
            for (int k = 0; k < 5; ++k) dst[k] = (double)res[k];
        }
    }
}

template <bool BF16, int MODE>
__global__ void __launch_bounds__(64) k_reduce_solve(IterCtx cx, SumSrc src, void* V, float* rv,
                                                     __nv_bfloat16* V3) {
    pdl_trigger();
    pdl_wait();
    reduce_solve_body<BF16, MODE>(cx, src, V, rv, V3, blockIdx.x, blockIdx.y);
}

// q1' = P1(q1) - c/rho - W and R1' = 2 P1(q1') - q1' - c/rho from W = A^T V;
// residual partials of the n-block (one per 128-row block and column).  The
// FP32 form's step after its cuBLAS GEMM2 (the BF16 forms run it in the
// tensor-core GEMM2 epilogue).  Grid (n_pad / 128, Kp), 128 threads.
template <bool BF16>
__global__ void __launch_bounds__(128) k_q1_update(IterCtx cx, SumSrc src, void* R1) {
    if (cx.ctrl->n_active == 0 || cx.ctrl->err) return;
    const int rt = blockIdx.x, p = rt * 128 + threadIdx.x, j = blockIdx.y;
    const bool check = is_check_iter(cx.ctrl, cx.check_every, cx.tol);
    const size_t o = (size_t)j * cx.n_pad + p;
    const int sl = cx.col_slot[p];
    Q1Update q = q1_update(cx.q1[o], gemm_out(src, p, j), u_at(cx, p, sl, j),
                           cx.c_slot[sl] * cx.inv_rho[j]);
    if (cx.active[j]) cx.q1[o] = q.qn;
    if (BF16) {
        __nv_bfloat16 hi, lo;
        split_bf16(q.r1, hi, lo);
        static_cast<__nv_bfloat16*>(R1)[o] = hi;
        static_cast<__nv_bfloat16*>(R1)[(size_t)cx.Kp * cx.n_pad + o] = lo;
    } else {
        static_cast<float*>(R1)[o] = q.r1;
    }
    if (check) {
        __shared__ double out[5];
        block_sum5(q.res, out);
        if (threadIdx.x == 0) {
            double* dst = cx.resid + ((size_t)rt * cx.Kp + j) * 5;
            for (int k = 0; k < 5; ++k) dst[k] = out[k];
        }
    }
}

// Per-column stop test and bookkeeping; the last kernel of every iteration.
// One block per column sums that column's residual partials (fixed order,
// deterministic); the last block to finish (ticket) updates the control
// block.
__device__ __forceinline__ void finalize_body(const IterCtx& cx) {
    Control* c = cx.ctrl;
    if (c->n_active == 0) return;
    const int it = c->iter + 1;
    __shared__ double red[5 * 4];
    finalize_column(cx, blockIdx.x, it, c->err != 0, red);
    // last block: count the active columns, advance the iteration counter
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&c->ticket, 1) == cx.Kp - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ int cnt;
    finalize_count(cx, it, &cnt);
}

__global__ void __launch_bounds__(128) k_finalize(IterCtx cx) {
    pdl_trigger();
    pdl_wait();
    finalize_body(cx);
}

// The element-wise kernels over the members of a group solve (run_group):
// one launch per step, member g = blockIdx.z, each member's own grid inside
// the launch's (the largest member's); the bodies are those above.
struct EwMember {
    IterCtx cx;
    SumSrc src;
    void* p0;               // rhs planes (reduce_rhs), V (reduce_solve), rhs planes (reduce_err)
    float* f1;              // rhs32 (reduce_rhs, reduce_err), rv (reduce_solve)
    __nv_bfloat16* b2;      // V3 (reduce_solve)
};
struct EwGroup {
    EwMember m[4];
    int G;
};

__device__ __forceinline__ const EwMember* ew_member(const EwGroup& P, int rows_per_block) {
    if ((int)blockIdx.z >= P.G) return nullptr;
    const EwMember& e = P.m[blockIdx.z];
    if ((int)blockIdx.x >= e.cx.m_pad / rows_per_block || (int)blockIdx.y >= e.cx.Kp) return nullptr;
    return &e;
}

__global__ void __launch_bounds__(64) k_reduce_rhs_g(const __grid_constant__ EwGroup P) {
    pdl_trigger();
    pdl_wait();
    if (const EwMember* e = ew_member(P, 256))
        reduce_rhs_body<true>(e->cx, e->src, e->p0, e->f1, blockIdx.x, blockIdx.y);
}

template <int MODE>
__global__ void __launch_bounds__(64) k_reduce_solve_g(const __grid_constant__ EwGroup P) {
    pdl_trigger();
    pdl_wait();
    if (const EwMember* e = ew_member(P, 256))
        reduce_solve_body<true, MODE>(e->cx, e->src, e->p0, e->f1, e->b2, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(64) k_reduce_err_g(const __grid_constant__ EwGroup P) {
    pdl_trigger();
    pdl_wait();
    if (const EwMember* e = ew_member(P, 256))
        reduce_err_body(e->cx, e->src, e->f1, static_cast<__nv_bfloat16*>(e->p0), blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(128) k_finalize_g(const __grid_constant__ EwGroup P) {
    pdl_trigger();
    pdl_wait();
    if ((int)blockIdx.z >= P.G) return;
    const EwMember& e = P.m[blockIdx.z];
    if ((int)blockIdx.x >= e.cx.Kp) return;
    finalize_body(e.cx);
}

// c^T z1 in FP64 per column (deterministic block reduction).
__global__ void k_objective(IterCtx cx, double* obj) {
    int j = blockIdx.x;
    __shared__ double red[256];
    double s = 0.0;
    for (int p = threadIdx.x; p < cx.n_pad; p += 256) {
        int sl = cx.col_slot[p];
        float u = u_at(cx, p, sl, j);
        float z = fminf(fmaxf(cx.q1[(size_t)j * cx.n_pad + p], 0.f), u);
        s += (double)cx.c_slot[sl] * (double)z;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) obj[j] = red[0];
}

// lambda = D_r * rho * y2 = D_r * rho * max(q2 - b, 0) (FP64), K x m.
__global__ void k_lambda(IterCtx cx, int K, double* lam) {
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= cx.m || j >= K) return;
    double q = cx.q2[(size_t)j * cx.m_pad + i];
    double bb = (double)b_of(i, j, cx.n_beams, cx.m, cx.Dr, cx.wbot);
    lam[(size_t)j * cx.m + i] = cx.Dr[i] * (double)cx.rho[j] * fmax(q - bb, 0.0);
}

// lambda (as k_lambda) of the listed columns: lam[c][m] for column cols[c].
__global__ void k_lambda_cols(IterCtx cx, const int* __restrict__ cols, double* lam) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
    if (i >= cx.m) return;
    const int j = cols[c];
    const double q = cx.q2[(size_t)j * cx.m_pad + i];
    const double bb = (double)b_of(i, j, cx.n_beams, cx.m, cx.Dr, cx.wbot);
    lam[(size_t)c * cx.m + i] = cx.Dr[i] * (double)cx.rho[j] * fmax(q - bb, 0.0);
}

// A column taken by a new weighting (streaming solve): q1 = q2 = 0, R1 from
// q1 = 0 under the column's new bounds (as k_init_r1), lagged low-term
// products zero until the column's first full iteration.
template <bool BF16>
__global__ void k_reset_cols(IterCtx cx, const int* __restrict__ cols, void* R1, float* c1, float* c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, j = cols[blockIdx.y];
    if (e < cx.n_pad) {
        const size_t o = (size_t)j * cx.n_pad + e;
        const int sl = cx.col_slot[e];
        const float u = u_at(cx, e, sl, j);
        const float r = 2.f * fminf(0.f, u) - cx.c_slot[sl] * cx.inv_rho[j];
        cx.q1[o] = 0.f;
        if (BF16) {
            __nv_bfloat16 hi, lo;
            split_bf16(r, hi, lo);
            static_cast<__nv_bfloat16*>(R1)[o] = hi;
            static_cast<__nv_bfloat16*>(R1)[(size_t)cx.Kp * cx.n_pad + o] = lo;
        } else {
            static_cast<float*>(R1)[o] = r;
        }
        if (c2) c2[o] = 0.f;
    }
    if (e < cx.m_pad) {
        const size_t o = (size_t)j * cx.m_pad + e;
        cx.q2[o] = 0.f;
        if (c1) c1[o] = 0.f;
    }
}

// Penalty change of the listed columns (residual balancing): rho_j was
// multiplied by f = fac[c] (colp already holds the new rho and 1/rho).  The
// projections z = P(q) stay, the scaled duals y = q - z become y / f (the
// multipliers rho y are unchanged), and R1 = 2 P1(q1) - q1 - c/rho is rebuilt
// for the next GEMM1 with the new q1 and rho.
template <bool BF16>
__global__ void k_rescale_cols(IterCtx cx, const int* __restrict__ cols, const float* __restrict__ fac,
                               void* R1) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y, j = cols[c];
    const float inv_f = 1.0f / fac[c];
    if (e < cx.n_pad) {
        const size_t o = (size_t)j * cx.n_pad + e;
        const int sl = cx.col_slot[e];
        const float u = u_at(cx, e, sl, j);
        const float q = cx.q1[o];
        const float z = fminf(fmaxf(q, 0.f), u);
        const float qn = z + (q - z) * inv_f;
        cx.q1[o] = qn;
        const float r = 2.f * z - qn - cx.c_slot[sl] * cx.inv_rho[j];
        if (BF16) {
            __nv_bfloat16 hi, lo;
            split_bf16(r, hi, lo);
            static_cast<__nv_bfloat16*>(R1)[o] = hi;
            static_cast<__nv_bfloat16*>(R1)[(size_t)cx.Kp * cx.n_pad + o] = lo;
        } else {
            static_cast<float*>(R1)[o] = r;
        }
    }
    if (e < cx.m_pad) {
        const size_t o = (size_t)j * cx.m_pad + e;
        const float q = cx.q2[o];
        const float z = fminf(q, b_of(e, j, cx.n_beams, cx.m, cx.Dr, cx.wbot));
        cx.q2[o] = z + (q - z) * inv_f;
    }
}

// q1 (K x n) and q2 (K x m) of the q-form state, FP64.
__global__ void k_state(IterCtx cx, int K, double* q1, double* q2) {
    int e = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (j >= K) return;
    if (q1 && e < cx.n) q1[(size_t)j * cx.n + e] = cx.q1[(size_t)j * cx.n_pad + e];
    if (q2 && e < cx.m) q2[(size_t)j * cx.m + e] = cx.q2[(size_t)j * cx.m_pad + e];
}

// ----------------------------------------------------------------- driver

static IterCtx make_ctx(ResultData& r) {
    CaseData& cs = *r.cs;
    IterCtx cx{};
    cx.Kp = r.Kp; cx.m = cs.m; cx.m_pad = cs.m_pad; cx.n_pad = cs.n_pad; cx.n_beams = cs.n_beams;
    cx.n_slot = cs.n_slot; cx.check_every = cs.prm.check_every; cx.max_iter = r.max_iter;
    cx.tol = (float)r.tol;
    cx.col_slot = cs.col_slot.as<uint8_t>();
    cx.utab = r.utab.as<float>();
    cx.mask = r.mask_words ? r.mask.as<uint32_t>() : nullptr;
    cx.c1 = r.refine ? r.c1.as<float>() : nullptr;
    cx.c2 = r.refine ? r.c2.as<float>() : nullptr;
    cx.mask_words = r.mask_words;
    cx.c_slot = r.utab.as<float>() + (size_t)r.Kp * cs.n_slot;
    cx.rho = r.colp.as<float>();
    cx.inv_rho = r.colp.as<float>() + r.Kp;
    cx.wbot = r.colp.as<float>() + 2 * r.Kp;
    cx.refine_on = r.colp.as<float>() + 3 * r.Kp;
    cx.Dr = cs.Dr.as<double>();
    cx.q1 = r.q1.as<float>(); cx.q2 = r.q2.as<float>();
    cx.active = r.active.as<int>(); cx.iters = r.iters.as<int>();
    cx.ctrl = r.ctrl.as<Control>();
    cx.resid = r.resid.as<double>();
    cx.stats = r.stats.as<double>();
    cx.n_resid_n = r.n_resid_n; cx.n_resid_m = r.n_resid_m;
    cx.eps_abs = cs.prm.eps_abs;
    cx.n = cs.n; cx.m_rows = cs.m;
    return cx;
}

IterCtx make_ctx_public(ResultData& r) { return make_ctx(r); }

static SumSrc plain_src(const float* p, int rows_pad) { return SumSrc{p, nullptr, nullptr, rows_pad, 0, 1, 1}; }

static SumSrc plan_src(const ResultData& r, const GemmPlan& P) {
    return SumSrc{r.part.as<float>(), P.tile_begin, P.tile_slots, 0, P.rows, P.n_tile, P.mt};
}

static int iteration_fp32(ResultData& r, const IterCtx& cx, int itx) {
    CaseData& cs = *r.cs;
    cudaStream_t st = cs.stream;
    const float one = 1.f, zero = 0.f;
    float* part = r.part.as<float>();
    prof_mark(r, itx, 0);
    // GEMM1: part[Kp][m_pad] = R1[Kp][n_pad] . A[m_pad][n_pad]^T
    if (cublasSgemm(cs.cublas, CUBLAS_OP_T, CUBLAS_OP_N, cs.m_pad, r.Kp, cs.n_pad, &one,
                    cs.A32.as<float>(), cs.n_pad, r.R1.as<float>(), cs.n_pad, &zero, part,
                    cs.m_pad) != CUBLAS_STATUS_SUCCESS) {
        set_error("cublasSgemm (GEMM1) failed");
        return LGK_ECUDA;
    }
    count_launch();
    prof_mark(r, itx, 1);
    dim3 gm(cs.m_pad / 256, r.Kp);
    k_reduce_rhs<false><<<gm, 64, 0, st>>>(cx, plain_src(part, cs.m_pad), r.rhs.p, nullptr);
    LGK_LAUNCH_CHECK();
    prof_mark(r, itx, 2);
    // solve: part = rhs . G^T (G symmetric)
    if (cublasSgemm(cs.cublas, CUBLAS_OP_T, CUBLAS_OP_N, cs.m_pad, r.Kp, cs.m_pad, &one,
                    cs.G32.as<float>(), cs.m_pad, r.rhs.as<float>(), cs.m_pad, &zero, part,
                    cs.m_pad) != CUBLAS_STATUS_SUCCESS) {
        set_error("cublasSgemm (solve) failed");
        return LGK_ECUDA;
    }
    count_launch();
    prof_mark(r, itx, 3);
    k_reduce_solve<false, RS_PLAIN><<<gm, 64, 0, st>>>(cx, plain_src(part, cs.m_pad), r.V.p, nullptr, nullptr);
    LGK_LAUNCH_CHECK();
    prof_mark(r, itx, 4);
    // GEMM2: W[Kp][n_pad] = V[Kp][m_pad] . A[m_pad][n_pad]
    if (cublasSgemm(cs.cublas, CUBLAS_OP_N, CUBLAS_OP_N, cs.n_pad, r.Kp, cs.m_pad, &one,
                    cs.A32.as<float>(), cs.n_pad, r.V.as<float>(), cs.m_pad, &zero,
                    r.W.as<float>(), cs.n_pad) != CUBLAS_STATUS_SUCCESS) {
        set_error("cublasSgemm (GEMM2) failed");
        return LGK_ECUDA;
    }
    count_launch();
    prof_mark(r, itx, 5);
    dim3 gn(cs.n_pad / 128, r.Kp);
    k_q1_update<false><<<gn, 128, 0, st>>>(cx, plain_src(r.W.as<float>(), cs.n_pad), r.R1.p);
    LGK_LAUNCH_CHECK();
    prof_mark(r, itx, 6);
    k_finalize<<<r.Kp, 128, 0, st>>>(cx);
    LGK_LAUNCH_CHECK();
    prof_mark(r, itx, 7);
    return LGK_OK;
}

// BF16 forms: GEMM1 and the solve leave stream-K partial sums that a reduce
// kernel adds (rhs, q2 steps); GEMM2 runs the q1 step in its own epilogue.
static int iteration_bf16(ResultData& r, const IterCtx& cx, int itx) {
    CaseData& cs = *r.cs;
    cudaStream_t st = cs.stream;
    int rc;
    dim3 gm(cs.m_pad / 256, r.Kp);
    // consecutive kernels overlap launch and set-up with the predecessor's
    // tail (programmatic dependent launch), except across profiling events
    const bool pdl = r.prof_ev.empty();
    // lo_refresh: the low term's products are recomputed on the solve's
    // first iteration and on every residual-test iteration, so each test sees
    // the two-term operator; in between they are reused.  The graph's first
    // slot carries the first iteration's refresh, skipped on the device in
    // later replays.
    const bool test_slot = (itx + 1) % cs.prm.check_every == 0;
    const bool full = r.refine && (itx == 0 || test_slot);
    const bool first_only = itx == 0 && !test_slot;
    int k = 0;                       // launch slot of this iteration (profile events)
    auto ran = [&](bool v) {
        if (!r.prof_ran.empty()) r.prof_ran[(size_t)itx * r.prof_class.size() + k] = v;
    };
    auto next = [&]() { prof_mark(r, itx, ++k); };
    prof_mark(r, itx, 0);
    if (full && (rc = tc_gemm1_lo(r, pdl && itx > 0, first_only))) return rc;
    ran(full);
    next();
    if ((rc = tc_gemm1(r, pdl && (itx > 0 || full)))) return rc;
    next();
    float* rhs32 = r.refine_steps ? r.rhs32.as<float>() : nullptr;
    __nv_bfloat16* V3 = r.refine_steps ? r.V3.as<__nv_bfloat16>() : nullptr;
    float* rv = r.refine_steps ? r.rv.as<float>() : nullptr;
    LGK_CUDA_TRY(launch_k(k_reduce_rhs<true>, gm, dim3(64), 0, st, pdl, cx, plan_src(r, r.plan1), r.rhs.p, rhs32));
    LGK_LAUNCH_CHECK();
    next();
    if ((rc = tc_solve(r, pdl))) return rc;
    next();
    if (r.refine_steps == 0) {
        LGK_CUDA_TRY(launch_k(k_reduce_solve<true, RS_PLAIN>, gm, dim3(64), 0, st, pdl, cx, plan_src(r, r.plan_s),
                              r.V.p, rv, V3));
    } else {
        LGK_CUDA_TRY(launch_k(k_reduce_solve<true, RS_FIRST>, gm, dim3(64), 0, st, pdl, cx, plan_src(r, r.plan_s),
                              r.V.p, rv, V3));
    }
    LGK_LAUNCH_CHECK();
    next();
    // refinement: e = rhs - S v, v += S^{-1} e
    for (int step = 1; step <= r.refine_steps; ++step) {
        if ((rc = tc_sv(r, pdl))) return rc;
        next();
        LGK_CUDA_TRY(launch_k(k_reduce_err, gm, dim3(64), 0, st, pdl, cx, plan_src(r, r.plan_s), rhs32,
                              r.rhs.as<__nv_bfloat16>()));
        LGK_LAUNCH_CHECK();
        next();
        if ((rc = tc_solve(r, pdl))) return rc;
        next();
        if (step < r.refine_steps) {
            LGK_CUDA_TRY(launch_k(k_reduce_solve<true, RS_ACCUM>, gm, dim3(64), 0, st, pdl, cx,
                                  plan_src(r, r.plan_s), r.V.p, rv, V3));
        } else {
            LGK_CUDA_TRY(launch_k(k_reduce_solve<true, RS_FINAL>, gm, dim3(64), 0, st, pdl, cx,
                                  plan_src(r, r.plan_s), r.V.p, rv, V3));
        }
        LGK_LAUNCH_CHECK();
        next();
    }
    if (full && (rc = tc_gemm2_lo(r, pdl, first_only))) return rc;
    ran(full);
    next();
    if ((rc = tc_gemm2(r, pdl))) return rc;
    next();
    LGK_CUDA_TRY(launch_k(k_finalize, dim3(r.Kp), dim3(128), 0, st, pdl, cx));
    LGK_LAUNCH_CHECK();
    next();
    return LGK_OK;
}

int run_solve(ResultData& r, const double* W, const double* rho, const double* q1_init,
              const double* q2_init, const uint32_t* mask, const StreamSpec* stream, bool prepare_only) {
    CaseData& cs = *r.cs;
    cudaStream_t st = cs.stream;
    const bool bf16 = cs.prm.precision != LGK_PREC_FP32;
    const int K = r.K;
    // column tiles: <= 256 columns each, multiples of 16 (tcgen05 N)
    int kp16 = (int)round_up(K, 16);
    int nt = (kp16 + 255) / 256;
    r.n_tile = (int)round_up((kp16 + nt - 1) / nt, 16);
    if (r.n_tile > 128) r.n_tile = (int)round_up(r.n_tile, 32);
    r.Kp = r.n_tile * nt;
    // the solve carries three B parts per stage: halve wide tiles
    r.n_tile_s = r.n_tile > 128 ? r.n_tile / 2 : r.n_tile;
    const int Kp = r.Kp, T = cs.n_targets, S = cs.n_slot;

    // point selection per column (second pass, Sec. 2.C): device layout
    // [n_pad][mw] words, rows past the points (BOT columns, padding) all set;
    // the point counts N_alpha that normalise u are the selected counts
    const int mw = (Kp + 31) / 32;
    std::vector<int> cnt((size_t)K * S);
    for (int j = 0; j < K; ++j) std::copy(cs.slot_count.begin(), cs.slot_count.end(), &cnt[(size_t)j * S]);
    std::vector<uint32_t> mdev;
    if (mask) {
        const int cw = (K + 31) / 32;
        mdev.assign((size_t)cs.n_pad * mw, 0xffffffffu);
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int p = 0; p < cs.n_pts; ++p) {
            uint32_t* row = &mdev[(size_t)p * mw];
            for (int w = 0; w < mw; ++w) row[w] = w < cw ? mask[(size_t)p * cw + w] : 0u;
            if (cw * 32 > K) row[cw - 1] &= (K % 32) ? ((1u << (K % 32)) - 1u) : 0xffffffffu;
            const int sl = cs.slot_host[p];
            for (int j = 0; j < K; ++j) cnt[(size_t)j * S + sl] += (row[j >> 5] >> (j & 31)) & 1u;
        }
    }
    r.mask_words = mask ? mw : 0;

    // per-column tables (Appendix A bounds; Eq. rho_rule or caller rho)
    std::vector<float> utab((size_t)Kp * S + S, 0.0f), colp((size_t)4 * Kp, 0.0f);
    r.u64.assign((size_t)Kp * S, 0.0);
    r.wb64.assign(Kp, 0.0);
    // column j's tables for weights w = (w_T, w_R, w_LD, w_BOT), penalty rh and
    // per-slot point counts nc
    auto fill_col = [&](int j, const double* w, double rh, const int* nc) {
        const double wT = w[0], wR = w[1], wLD = w[2], wB = w[3];
        double* u = &r.u64[(size_t)j * S];
        for (int k = 0; k < T; ++k) {
            u[3 * k] = nc[3 * k] ? cs.q_area[k] * wT / nc[3 * k] : 0.0;
            u[3 * k + 1] = nc[3 * k + 1] ? cs.q_vol[k] * wT / nc[3 * k + 1] : 0.0;
            u[3 * k + 2] = nc[3 * k + 2] ? (wR / T) / nc[3 * k + 2] : 0.0;
        }
        u[slot_ld1(T)] = nc[slot_ld1(T)] ? wLD / nc[slot_ld1(T)] : 0.0;
        u[slot_ld2(T)] = nc[slot_ld2(T)] ? wLD / nc[slot_ld2(T)] : 0.0;
        u[slot_oar(T)] = INFINITY;
        u[slot_bot(T)] = INFINITY;
        u[slot_pad(T)] = 0.0;
        for (int s = 0; s < S; ++s) utab[(size_t)j * S + s] = (float)u[s];
        r.wb64[j] = wB;
        colp[j] = (float)rh;
        colp[Kp + j] = (float)(1.0 / rh);
        colp[2 * Kp + j] = (float)wB;
        colp[3 * Kp + j] = cs.prm.solve_refine > 0 ? 1.0f : 0.0f;   // refined from the start, or by age
    };
    for (int j = 0; j < K; ++j) fill_col(j, W + 4 * (size_t)j, rho[j], &cnt[(size_t)j * S]);
    for (int s = 0; s < S; ++s) utab[(size_t)Kp * S + s] = cs.c_of_slot[s];

    // buffers
    int rc;
    const size_t nq = (size_t)Kp * cs.n_pad, mq = (size_t)Kp * cs.m_pad;
    if ((rc = r.q1.alloc(nq * 4)) || (rc = r.q2.alloc(mq * 4))) return rc;
    if ((rc = r.R1.alloc(bf16 ? nq * 4 : nq * 4))) return rc;     // 2 x bf16 or 1 x f32
    if ((rc = r.rhs.alloc(bf16 ? mq * 6 : mq * 4)) || (rc = r.V.alloc(mq * 4))) return rc;
    if (!bf16 && (rc = r.W.alloc(nq * 4))) return rc;
    if (!bf16 && (rc = r.part.alloc(mq * 4))) return rc;     // BF16 forms: tc_prepare
    if ((rc = r.utab.alloc(utab.size() * 4)) || (rc = r.colp.alloc(colp.size() * 4))) return rc;
    r.refine = cs.na == 2 && cs.prm.lo_refresh;
    r.refine_steps = bf16 && cs.S3.p ? cs.prm.solve_refine : 0;
    if (r.refine_steps) {
        if ((rc = r.rhs32.alloc(mq * 4)) || (rc = r.rv.alloc(mq * 4)) || (rc = r.V3.alloc(mq * 6))) return rc;
    }
    // S^{-1} kept in L2 across iterations (lgk_params.l2_keep_inverse): a
    // persisting carve-out of the L2 (a setting of this process's context,
    // released when the solve ends) and an access-policy window over the
    // inverse's terms on the solve's launches, which load it evict-last
    struct L2Release {
        ResultData& r;
        ~L2Release() {
            if (!r.l2_keep) return;
            cudaCtxResetPersistingL2Cache();
            cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0);
            cudaGetLastError();
            r.l2_keep = false;
        }
    } l2_release{r};
    r.l2_keep = false;
    if (bf16 && cs.prm.l2_keep_inverse && cs.G3.p && !prepare_only) {
        int max_keep = 0, max_win = 0;
        if (cudaDeviceGetAttribute(&max_keep, cudaDevAttrMaxPersistingL2CacheSize, cs.device) == cudaSuccess &&
            cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, cs.device) == cudaSuccess &&
            max_keep > 0 && max_win > 0) {
            const size_t win = std::min(cs.G3.bytes, (size_t)max_win);
            const size_t keep = std::min(win, (size_t)max_keep);
            if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, keep) == cudaSuccess) {
                r.l2win = cudaAccessPolicyWindow{};
                r.l2win.base_ptr = cs.G3.p;
                r.l2win.num_bytes = win;
                r.l2win.hitRatio = (float)((double)keep / (double)win);
                r.l2win.hitProp = cudaAccessPropertyPersisting;
                r.l2win.missProp = cudaAccessPropertyStreaming;
                r.l2_keep = true;
            }
        }
        cudaGetLastError();
    }
    if (r.refine) {
        if ((rc = r.c1.alloc(mq * 4)) || (rc = r.c2.alloc(nq * 4))) return rc;
        LGK_CUDA_TRY(cudaMemsetAsync(r.c1.p, 0, r.c1.bytes, st));
        LGK_CUDA_TRY(cudaMemsetAsync(r.c2.p, 0, r.c2.bytes, st));
    }
    if (mask && (rc = r.mask.alloc(mdev.size() * 4))) return rc;
    if ((rc = r.active.alloc((size_t)2 * Kp * 4)) || (rc = r.iters.alloc((size_t)Kp * 4))) return rc;
    if ((rc = r.ctrl.alloc(sizeof(Control)))) return rc;
    r.n_resid_n = cs.n_pad / 128;
    r.n_resid_m = cs.m_pad / 128;
    if ((rc = r.resid.alloc((size_t)(r.n_resid_n + r.n_resid_m) * Kp * 5 * 8))) return rc;
    if ((rc = r.stats.alloc((size_t)3 * Kp * 8))) return rc;
    // iterations per captured graph (one replay)
    const int per_graph = std::max(1, std::min(r.max_iter, 5 * cs.prm.check_every));
    // streaming: the weighting (tag) each column holds (-1: none), the
    // iteration it started at, the next weighting to admit.  A dynamic
    // stream's counter starts at one replay, so no column gets the first-
    // iteration refresh of the lagged products: every column, initial or
    // refilled, runs the same iteration from its own start.
    const bool dynamic = stream && stream->pull;
    const int n0 = stream && stream->n_initial >= 0 ? std::min(stream->n_initial, K) : K;
    const int iter0 = dynamic ? per_graph : 0;
    std::vector<long long> tag_of;
    std::vector<int> start_it;
    int next_w = K;
    DevBuf cols_d, lam_d;
    if (stream) {
        tag_of.assign(Kp, -1);
        start_it.assign(Kp, iter0);
        for (int j = 0; j < n0; ++j) tag_of[j] = stream->initial_tags ? stream->initial_tags[j] : j;
        if ((rc = cols_d.alloc((size_t)Kp * 4)) || (rc = lam_d.alloc((size_t)Kp * cs.m * 8))) return rc;
    }

    std::vector<int> act(2 * Kp, 0);
    for (int j = 0; j < n0; ++j) act[j] = 1;
    Control c0{iter0, n0, r.max_iter, 0, 0};
    LGK_CUDA_TRY(cudaMemcpyAsync(r.utab.p, utab.data(), utab.size() * 4, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(r.colp.p, colp.data(), colp.size() * 4, cudaMemcpyHostToDevice, st));
    if (mask)
        LGK_CUDA_TRY(cudaMemcpyAsync(r.mask.p, mdev.data(), mdev.size() * 4, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(r.active.p, act.data(), act.size() * 4, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(r.ctrl.p, &c0, sizeof(c0), cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemsetAsync(r.iters.p, 0, r.iters.bytes, st));
    LGK_CUDA_TRY(cudaMemsetAsync(r.q1.p, 0, r.q1.bytes, st));
    LGK_CUDA_TRY(cudaMemsetAsync(r.q2.p, 0, r.q2.bytes, st));
    std::vector<float> init_buf;
    if (q1_init) {       // warm start / resume: K x n FP64 -> [Kp][n_pad] FP32
        init_buf.assign((size_t)Kp * cs.n_pad, 0.0f);
        for (int j = 0; j < K; ++j)
            for (int p = 0; p < cs.n; ++p) init_buf[(size_t)j * cs.n_pad + p] = (float)q1_init[(size_t)j * cs.n + p];
        LGK_CUDA_TRY(cudaMemcpyAsync(r.q1.p, init_buf.data(), init_buf.size() * 4, cudaMemcpyHostToDevice, st));
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (q2_init) {
        init_buf.assign((size_t)Kp * cs.m_pad, 0.0f);
        for (int j = 0; j < K; ++j)
            for (int i = 0; i < cs.m; ++i) init_buf[(size_t)j * cs.m_pad + i] = (float)q2_init[(size_t)j * cs.m + i];
        LGK_CUDA_TRY(cudaMemcpyAsync(r.q2.p, init_buf.data(), init_buf.size() * 4, cudaMemcpyHostToDevice, st));
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
    }
    LGK_CUDA_TRY(cudaMemsetAsync(r.stats.p, 0, r.stats.bytes, st));
    LGK_CUDA_TRY(cudaMemsetAsync(r.resid.p, 0, r.resid.bytes, st));

    IterCtx cx = make_ctx(r);
    {
        dim3 g((cs.n_pad + 255) / 256, Kp);
        if (bf16) k_init_r1<true><<<g, 256, 0, st>>>(cx, r.R1.p);
        else k_init_r1<false><<<g, 256, 0, st>>>(cx, r.R1.p);
        LGK_LAUNCH_CHECK();
    }
    // GEMM configurations (lgk_params.autotune): the case's stored choice for
    // this column count, or candidates to time on the first replays
    std::vector<std::pair<int, int>> cands;
    size_t tune_next = 0;
    std::vector<float> tune_ms;
    if (bf16 && cs.prm.autotune && !prepare_only) {
        std::lock_guard<std::mutex> lk(cs.tune_mu);
        auto it = cs.tuned.find(Kp);
        if (it != cs.tuned.end()) {
            r.force_wide = it->second.first & 1;
            r.force_wide2 = (it->second.first >> 1) & 1;
            r.n_tile_s = it->second.second;
        } else {
            // candidates: 256- or 128-row tiles for GEMM1 (bit 0) and for
            // GEMM2 (bit 1) where the one-term A operand allows them, x the
            // solve's column tile whole or halved; the first is the default
            const bool can_wide = (cs.na == 1 || r.refine) && r.n_tile <= 128;
            std::vector<int> ws = can_wide ? std::vector<int>{3, 1, 2, 0} : std::vector<int>{0};
            std::vector<int> ss{r.n_tile_s};
            if (r.n_tile_s % 32 == 0) ss.push_back(r.n_tile_s / 2);
            for (int w : ws)
                for (int t : ss) cands.push_back({w, t});
            r.force_wide = cands[0].first & 1;
            r.force_wide2 = (cands[0].first >> 1) & 1;
            r.n_tile_s = cands[0].second;
        }
    }
    if (bf16) {
        if ((rc = tc_prepare(r))) return rc;
    } else {
        cublasSetStream(cs.cublas, st);
    }
    // a group solve (run_group) takes over from here with its own graph
    if (prepare_only) {
        r.colp_h = colp;
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
        return LGK_OK;
    }

    // capture a CUDA graph of `per_graph` iterations, replay until done
    cudaGraph_t g = nullptr;
    // kernel classes of one iteration, in launch order (again when the
    // iteration changes form: refine_after)
    size_t kpi = 0;
    auto prof_init = [&]() -> int {
        if (bf16) {
            r.prof_class = {LGK_K_GEMM1_LO, LGK_K_GEMM1, LGK_K_REDUCE_RHS, LGK_K_SOLVE, LGK_K_REDUCE_SOLVE};
            for (int step = 0; step < r.refine_steps; ++step)
                r.prof_class.insert(r.prof_class.end(),
                                    {LGK_K_SV, LGK_K_REDUCE_ERR, LGK_K_SOLVE, LGK_K_REDUCE_SOLVE});
            r.prof_class.insert(r.prof_class.end(), {LGK_K_GEMM2_LO, LGK_K_GEMM2, LGK_K_FINALIZE});
        } else {
            r.prof_class = {LGK_K_GEMM1, LGK_K_REDUCE_RHS, LGK_K_SOLVE, LGK_K_REDUCE_SOLVE,
                            LGK_K_GEMM2, LGK_K_Q1_UPDATE, LGK_K_FINALIZE};
        }
        kpi = r.prof_class.size();
        if (cs.prm.profile) {
            for (cudaEvent_t e : r.prof_ev)
                if (e) cudaEventDestroy(e);
            r.prof_ev.assign((size_t)per_graph * (kpi + 1), nullptr);
            for (auto& e : r.prof_ev) LGK_CUDA_TRY(cudaEventCreate(&e));
            r.prof_ran.assign((size_t)per_graph * kpi, 1);
        }
        return LGK_OK;
    };
    if ((rc = prof_init())) return rc;
    size_t n_nodes = 0;
    // capture the graph of `per_graph` iterations with the current ctx
    auto capture = [&]() -> int {
        LGK_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int it = 0; it < per_graph; ++it) {
            int rc2 = bf16 ? iteration_bf16(r, cx, it) : iteration_fp32(r, cx, it);
            if (rc2) {
                cudaStreamEndCapture(st, &g);
                if (g) cudaGraphDestroy(g);
                return rc2;
            }
        }
        LGK_CUDA_TRY(cudaStreamEndCapture(st, &g));
        // kernels per replay: the graph's kernel nodes (the captured launches
        // were counted at capture time, when nothing ran)
        size_t n_all = 0;
        n_nodes = 0;
        if (cudaGraphGetNodes(g, nullptr, &n_all) == cudaSuccess && n_all) {
            std::vector<cudaGraphNode_t> nodes(n_all);
            if (cudaGraphGetNodes(g, nodes.data(), &n_all) == cudaSuccess)
                for (auto nd : nodes) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++n_nodes;
                }
        }
        count_launch(-(long long)n_nodes);
        cudaError_t e = cudaGraphInstantiate(&r.graph, g, 0);
        cudaGraphDestroy(g);
        g = nullptr;
        if (e != cudaSuccess) {
            set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
            return LGK_ECUDA;
        }
        return LGK_OK;
    };
    if ((rc = capture())) return rc;
    r.graph_iters = per_graph;

    Control* hc = nullptr;
    LGK_CUDA_TRY(cudaMallocHost(&hc, sizeof(Control)));
    // streaming, at a replay boundary (the device idle): copy out the results
    // of the columns that stopped (their test passed, or their own iteration
    // cap), give those columns the next weightings, and push the new flags,
    // tables and counters.  done: no column holds a weighting; age: the
    // iterations of the oldest running column.
    // FP64 checks of a stream's stopped weightings (StreamSpec::check): their
    // states are saved at the boundary where they stop and checked in
    // batches of kChkSave (one pass over A per batch instead of one per
    // boundary)
    constexpr int kChkSave = 64;
    std::vector<long long> pend_tag;
    std::vector<float> pend_uf, pend_rho, pend_wbf;
    std::vector<double> pend_u64, pend_wb64;
    DevBuf saved;
    if (stream && stream->check &&
        (rc = saved.alloc((size_t)kChkSave * (cs.n_pad + cs.m_pad) * 4)))
        return rc;
    auto flush_checks = [&]() -> int {
        const int nc = (int)pend_tag.size();
        if (!nc) return LGK_OK;
        std::vector<int> src(nc);
        for (int c = 0; c < nc; ++c) src[c] = c;
        std::vector<double> out((size_t)nc * LGK_CHECK_COUNT);
        const int rcc = run_check_states(r, saved.as<float>(), saved.as<float>() + (size_t)kChkSave * cs.n_pad,
                                         nc, src.data(), nullptr, pend_uf.data(), pend_rho.data(),
                                         pend_wbf.data(), pend_u64.data(), pend_wb64.data(), out.data());
        if (rcc) return rcc;
        for (int c = 0; c < nc; ++c)
            std::copy(&out[(size_t)c * LGK_CHECK_COUNT], &out[(size_t)(c + 1) * LGK_CHECK_COUNT],
                      stream->check + (size_t)pend_tag[c] * LGK_CHECK_COUNT);
        pend_tag.clear();
        pend_uf.clear();
        pend_rho.clear();
        pend_wbf.clear();
        pend_u64.clear();
        pend_wb64.clear();
        return LGK_OK;
    };
    // the next weighting of the stream: from the caller's arrays, or pulled
    // from a dynamic source (1: one, 0: none now, -1: closed and drained)
    auto next_weighting = [&](double* w, double* rh, long long* tag, bool block) -> int {
        const StreamSpec& ss = *stream;
        if (ss.pull) return ss.pull(w, rh, tag, block);
        if (next_w >= ss.K_total) return -1;
        std::copy(ss.W + 4 * (size_t)next_w, ss.W + 4 * (size_t)next_w + 4, w);
        *rh = ss.rho[next_w];
        *tag = next_w++;
        return 1;
    };
    auto emit = [&](long long tag, const StreamOut& o) {
        const StreamSpec& ss = *stream;
        if (ss.done) {
            ss.done(tag, o);
            return;
        }
        const size_t w = (size_t)tag;
        if (ss.iters) ss.iters[w] = o.iters;
        if (ss.obj) ss.obj[w] = o.obj;
        if (ss.rel_pri) ss.rel_pri[w] = o.rel_pri;
        if (ss.rel_dual) ss.rel_dual[w] = o.rel_dual;
        if (ss.converged) ss.converged[w] = (uint8_t)o.converged;

        if (ss.t) std::copy(o.t, o.t + cs.n_beams, ss.t + w * cs.n_beams);
        if (ss.tau) std::copy(o.tau, o.tau + cs.n_iso, ss.tau + w * cs.n_iso);
    };
    // streaming, at a replay boundary (the device idle): copy out the results
    // of the columns that stopped (their test passed, or their own iteration
    // cap), give every free column the next weighting, and push the new
    // flags, tables and counters.  A dynamic stream with no weighting left in
    // any column waits here for the next one (its counter restarts).  done:
    // no column holds a weighting and none will come; age: the iterations of
    // the oldest running column.
    auto stream_boundary = [&](bool& done, int& age) -> int {
        const StreamSpec& ss = *stream;
        std::vector<int> a(2 * (size_t)Kp), its(Kp);
        LGK_CUDA_TRY(cudaMemcpyAsync(a.data(), r.active.p, a.size() * 4, cudaMemcpyDeviceToHost, st));
        LGK_CUDA_TRY(cudaMemcpyAsync(its.data(), r.iters.p, its.size() * 4, cudaMemcpyDeviceToHost, st));
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<int> ret;
        for (int j = 0; j < Kp; ++j) {
            if (tag_of[j] < 0) continue;
            if (a[j] && hc->iter - start_it[j] >= ss.max_iter) a[j] = 0;
            if (!a[j]) ret.push_back(j);
        }
        bool changed = false;
        if (!ret.empty()) {
            changed = true;
            k_objective<<<Kp, 256, 0, st>>>(cx, r.stats.as<double>() + 2 * Kp);
            LGK_LAUNCH_CHECK();
            LGK_CUDA_TRY(cudaMemcpyAsync(cols_d.p, ret.data(), ret.size() * 4, cudaMemcpyHostToDevice, st));
            k_lambda_cols<<<dim3((cs.m + 255) / 256, (unsigned)ret.size()), 256, 0, st>>>(
                cx, cols_d.as<int>(), lam_d.as<double>());
            LGK_LAUNCH_CHECK();
            std::vector<double> stv(3 * (size_t)Kp), lam(ret.size() * (size_t)cs.m);
            LGK_CUDA_TRY(cudaMemcpyAsync(stv.data(), r.stats.p, stv.size() * 8, cudaMemcpyDeviceToHost, st));
            LGK_CUDA_TRY(cudaMemcpyAsync(lam.data(), lam_d.p, lam.size() * 8, cudaMemcpyDeviceToHost, st));
            LGK_CUDA_TRY(cudaStreamSynchronize(st));
            std::vector<double> chk;
            r.colp_h = colp;
            if (ss.want_check && !ss.check) {  // FP64 check now, for the result callback
                chk.resize(ret.size() * (size_t)LGK_CHECK_COUNT);
                const int rcc = run_check(r, ret.data(), (int)ret.size(), chk.data());
                if (rcc) return rcc;
            }
            if (ss.check) {                    // save the state for a batched FP64 check
                for (int j : ret) {
                    if ((int)pend_tag.size() == kChkSave) {
                        const int rcf = flush_checks();
                        if (rcf) return rcf;
                    }
                    const int slot = (int)pend_tag.size();
                    LGK_CUDA_TRY(cudaMemcpyAsync(saved.as<float>() + (size_t)slot * cs.n_pad,
                                                 r.q1.as<float>() + (size_t)j * cs.n_pad, (size_t)cs.n_pad * 4,
                                                 cudaMemcpyDeviceToDevice, st));
                    LGK_CUDA_TRY(cudaMemcpyAsync(saved.as<float>() + (size_t)kChkSave * cs.n_pad +
                                                     (size_t)slot * cs.m_pad,
                                                 r.q2.as<float>() + (size_t)j * cs.m_pad, (size_t)cs.m_pad * 4,
                                                 cudaMemcpyDeviceToDevice, st));
                    pend_tag.push_back(tag_of[j]);
                    for (int sl = 0; sl < S; ++sl) {
                        pend_uf.push_back(utab[(size_t)j * S + sl]);
                        pend_u64.push_back(r.u64[(size_t)j * S + sl]);
                    }
                    pend_rho.push_back(colp[j]);
                    pend_wbf.push_back(colp[2 * (size_t)Kp + j]);
                    pend_wb64.push_back(r.wb64[j]);
                }
            }
            for (size_t c = 0; c < ret.size(); ++c) {
                const int j = ret[c];
                const double* l = &lam[c * (size_t)cs.m];
                StreamOut o{l, l + cs.n_beams, its[j] - start_it[j], stv[2 * (size_t)Kp + j], stv[j],
                            stv[(size_t)Kp + j], a[(size_t)Kp + j] != 0,
                            chk.empty() ? nullptr : &chk[c * LGK_CHECK_COUNT]};
                emit(tag_of[j], o);
                tag_of[j] = -1;
            }
        }
        // give every free column the next weighting
        std::vector<int> fill;
        bool closed = false;
        auto take = [&](int j, bool block) -> bool {
            double w[4], rh;
            long long tag;
            const int got = next_weighting(w, &rh, &tag, block);
            if (got < 0) closed = true;
            if (got != 1) return false;
            tag_of[j] = tag;
            fill_col(j, w, rh, cs.slot_count.data());
            a[j] = 1;
            a[(size_t)Kp + j] = 0;
            fill.push_back(j);
            return true;
        };
        // (the stream's width is K columns; the padding columns up to Kp stay empty)
        for (int j = 0; j < K && !closed; ++j)
            if (tag_of[j] < 0 && !take(j, false)) break;
        bool any = false;
        for (int j = 0; j < Kp; ++j) any = any || tag_of[j] >= 0;
        if (!any && dynamic && !closed) {
            // idle: wait for the next weighting; the counter restarts at one replay
            hc->iter = iter0;
            if (take(0, true))
                for (int j = 1; j < K && !closed; ++j)
                    if (!take(j, false)) break;
            changed = true;
        }
        if (changed) {
            // graph slots assume replays that start on a multiple of their length
            hc->iter = (int)round_up(hc->iter, per_graph);
            for (int j : fill) start_it[j] = hc->iter;
            if (!fill.empty()) {
                LGK_CUDA_TRY(cudaMemcpyAsync(r.utab.p, utab.data(), utab.size() * 4, cudaMemcpyHostToDevice, st));
                LGK_CUDA_TRY(cudaMemcpyAsync(r.colp.p, colp.data(), colp.size() * 4, cudaMemcpyHostToDevice, st));
                LGK_CUDA_TRY(cudaMemcpyAsync(cols_d.p, fill.data(), fill.size() * 4, cudaMemcpyHostToDevice, st));
                const int ne = std::max(cs.n_pad, cs.m_pad);
                dim3 g((ne + 255) / 256, (unsigned)fill.size());
                float* c1 = r.refine ? r.c1.as<float>() : nullptr;
                float* c2 = r.refine ? r.c2.as<float>() : nullptr;
                if (bf16) k_reset_cols<true><<<g, 256, 0, st>>>(cx, cols_d.as<int>(), r.R1.p, c1, c2);
                else k_reset_cols<false><<<g, 256, 0, st>>>(cx, cols_d.as<int>(), r.R1.p, c1, c2);
                LGK_LAUNCH_CHECK();
            }
            int n_act = 0;
            for (int j = 0; j < Kp; ++j) n_act += a[j] != 0;
            hc->n_active = n_act;
            LGK_CUDA_TRY(cudaMemcpyAsync(r.active.p, a.data(), a.size() * 4, cudaMemcpyHostToDevice, st));
            LGK_CUDA_TRY(cudaMemcpyAsync(r.ctrl.p, hc, sizeof(Control), cudaMemcpyHostToDevice, st));
            LGK_CUDA_TRY(cudaStreamSynchronize(st));
        }
        done = true;
        age = 0;
        for (int j = 0; j < Kp; ++j)
            if (tag_of[j] >= 0) {
                done = false;
                age = std::max(age, hc->iter - start_it[j]);
            }
        return LGK_OK;
    };
    // residual balancing (lgk_params.rho_adapt) at a replay boundary: columns
    // still running whose last residual test is this replay's get rho x 1.5
    // or / 1.5 when one relative residual exceeds 3 times the other (at most
    // 40 changes per column; a column refilled by a stream starts afresh)
    std::vector<int> rho_changes(Kp, 0), adapt_start(Kp, -1);
    DevBuf adapt_d;
    auto adapt_rho = [&]() -> int {
        std::vector<int> a(Kp);
        std::vector<double> stv(2 * (size_t)Kp);
        LGK_CUDA_TRY(cudaMemcpyAsync(a.data(), r.active.p, (size_t)Kp * 4, cudaMemcpyDeviceToHost, st));
        LGK_CUDA_TRY(cudaMemcpyAsync(stv.data(), r.stats.p, stv.size() * 8, cudaMemcpyDeviceToHost, st));
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<int> cols;
        std::vector<float> fac;
        for (int j = 0; j < Kp; ++j) {
            if (!a[j]) continue;
            const int start = stream ? start_it[j] : 0;
            if (adapt_start[j] != start) {          // a new weighting in this column
                adapt_start[j] = start;
                rho_changes[j] = 0;
            }
            if (hc->iter <= start || rho_changes[j] >= 40) continue;   // no test of its own yet
            const double rp = stv[j], rd = stv[(size_t)Kp + j];
            float f;
            if (rp > 3.0 * rd) f = 1.5f;
            else if (rd > 3.0 * rp) f = 1.0f / 1.5f;
            else continue;
            colp[j] *= f;
            colp[(size_t)Kp + j] = 1.0f / colp[j];
            ++rho_changes[j];
            cols.push_back(j);
            fac.push_back(f);
        }
        if (cols.empty()) return LGK_OK;
        r.colp_h = colp;
        if (!adapt_d.p) {
            const int rc2 = adapt_d.alloc((size_t)Kp * 8);
            if (rc2) return rc2;
        }
        int* cols_a = adapt_d.as<int>();
        float* fac_a = reinterpret_cast<float*>(cols_a + Kp);
        LGK_CUDA_TRY(cudaMemcpyAsync(r.colp.p, colp.data(), (size_t)2 * Kp * 4, cudaMemcpyHostToDevice, st));
        LGK_CUDA_TRY(cudaMemcpyAsync(cols_a, cols.data(), cols.size() * 4, cudaMemcpyHostToDevice, st));
        LGK_CUDA_TRY(cudaMemcpyAsync(fac_a, fac.data(), fac.size() * 4, cudaMemcpyHostToDevice, st));
        const int ne = std::max(cs.n_pad, cs.m_pad);
        dim3 g((ne + 255) / 256, (unsigned)cols.size());
        if (bf16) k_rescale_cols<true><<<g, 256, 0, st>>>(cx, cols_a, fac_a, r.R1.p);
        else k_rescale_cols<false><<<g, 256, 0, st>>>(cx, cols_a, fac_a, r.R1.p);
        LGK_LAUNCH_CHECK();
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
        return LGK_OK;
    };
    // a new GEMM configuration: re-plan and re-capture between two replays
    auto reconfigure = [&](int wide, int nts) -> int {
        cudaGraphExecDestroy(r.graph);
        r.graph = nullptr;
        r.force_wide = wide & 1;
        r.force_wide2 = (wide >> 1) & 1;
        r.n_tile_s = nts;
        int rc2 = tc_prepare(r);
        if (rc2) return rc2;
        cx = make_ctx(r);
        return capture();
    };
    cudaEvent_t tev[2] = {nullptr, nullptr};
    if (!cands.empty()) {
        LGK_CUDA_TRY(cudaEventCreate(&tev[0]));
        LGK_CUDA_TRY(cudaEventCreate(&tev[1]));
    }
    int iter_before = 0;
    auto t0 = std::chrono::steady_clock::now();
    rc = LGK_OK;
    for (;;) {
        if (dynamic) t0 = std::chrono::steady_clock::now();     // a server stream: bound each replay
        const bool timing = tune_next < cands.size();
        if (timing) cudaEventRecord(tev[0], st);
        cudaError_t le = cudaGraphLaunch(r.graph, st);
        if (timing) cudaEventRecord(tev[1], st);
        if (le != cudaSuccess) { set_error(cudaGetErrorString(le)); rc = LGK_ECUDA; break; }
        count_launch((long long)n_nodes - 0);
        cudaMemcpyAsync(hc, r.ctrl.p, sizeof(Control), cudaMemcpyDeviceToHost, st);
        for (;;) {
            cudaError_t q = cudaStreamQuery(st);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) { set_error(cudaGetErrorString(q)); rc = LGK_ECUDA; break; }
            auto el = std::chrono::steady_clock::now() - t0;
            if (std::chrono::duration_cast<std::chrono::milliseconds>(el).count() > cs.prm.timeout_ms) {
                set_error("solve exceeded timeout_ms");
                rc = LGK_ETIMEOUT;
                break;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        if (rc) break;
        if (hc->err) {
            set_error("device error flag " + std::to_string(hc->err) + " raised during the solve");
            rc = LGK_ECUDA;
            break;
        }
        if (r.cancel.load()) {
            set_error("solve cancelled (its result was freed while it ran)");
            rc = LGK_ETIMEOUT;
            break;
        }
        if (!r.prof_ev.empty()) {       // iterations of this replay that did work
            int worked = std::min(per_graph, hc->iter - iter_before);
            for (int it = 0; it < worked; ++it)
                for (size_t k = 0; k < kpi; ++k) {
                    float ms = 0.f;
                    const size_t e0 = (size_t)it * (kpi + 1) + k;
                    if (!r.prof_ran[(size_t)it * kpi + k]) continue;      // slot without a kernel
                    if (cudaEventElapsedTime(&ms, r.prof_ev[e0], r.prof_ev[e0 + 1]) == cudaSuccess) {
                        r.prof_ms[r.prof_class[k]] += ms;
                        r.prof_n[r.prof_class[k]] += 1;
                    } else {
                        cudaGetLastError();      // not sticky; keep it out of later checks
                    }
                }
        }
        iter_before = hc->iter;
        int age = hc->iter;         // iterations of the oldest running column
        if (stream) {
            bool done = false;
            if ((rc = stream_boundary(done, age))) break;
            if (done) break;
            iter_before = hc->iter;
        } else if (hc->n_active == 0) {
            break;
        }
        if (cs.prm.rho_adapt && (rc = adapt_rho())) break;
        if (timing) {
            // autotuner: this replay ran candidate tune_next; time the next one,
            // or keep the fastest (ties: the earlier, i.e. the default) for
            // this case and column count
            float ms = 0.f;
            cudaEventElapsedTime(&ms, tev[0], tev[1]);
            tune_ms.push_back(ms);
            ++tune_next;
            std::pair<int, int> pick = cands[tune_next < cands.size() ? tune_next : 0];
            if (tune_next == cands.size()) {
                size_t best = 0;
                for (size_t c = 1; c < tune_ms.size(); ++c)
                    if (tune_ms[c] < tune_ms[best]) best = c;
                pick = cands[best];
                std::lock_guard<std::mutex> lk(cs.tune_mu);
                cs.tuned[Kp] = pick;
            }
            if ((pick.first != (r.force_wide | (r.force_wide2 << 1)) || pick.second != r.n_tile_s) &&
                (rc = reconfigure(pick.first, pick.second)))
                break;
        }
        if (r.refine && cs.prm.lo_refresh_iters > 0 && age >= cs.prm.lo_refresh_iters) {
            // columns still running this long: continue with the literal
            // iteration (all terms every step) from the current state
            cudaGraphExecDestroy(r.graph);
            r.graph = nullptr;
            r.refine = false;
            if ((rc = tc_prepare(r))) break;
            cx = make_ctx(r);
            if ((rc = capture())) break;
        }
        if (bf16 && r.refine_steps == 0 && cs.S3.p && cs.prm.refine_after > 0 && age >= cs.prm.refine_after) {
            // columns still running this long: continue with one refinement
            // step of the solve per iteration (their residuals may have
            // levelled off at the unrefined solve's accuracy floor)
            cudaGraphExecDestroy(r.graph);
            r.graph = nullptr;
            const size_t mq2 = (size_t)Kp * cs.m_pad;
            if ((rc = r.rhs32.alloc(mq2 * 4)) || (rc = r.rv.alloc(mq2 * 4)) || (rc = r.V3.alloc(mq2 * 6))) break;
            r.refine_steps = 1;
            if ((rc = prof_init())) break;
            if ((rc = tc_prepare(r))) break;
            cx = make_ctx(r);
            if ((rc = capture())) break;
        }
        if (r.refine_steps > 0 && cs.prm.solve_refine == 0) {
            // refine_after applies per column, by the column's own age, so a
            // weighting's arithmetic does not depend on what else runs beside
            // it (a stream refills columns; a younger column keeps e = 0)
            bool flip = false;
            for (int j = 0; j < Kp; ++j) {
                const bool holds = stream ? tag_of[j] >= 0 : j < K;
                const int own = hc->iter - (stream ? start_it[j] : 0);
                const float on = holds && own >= cs.prm.refine_after ? 1.0f : 0.0f;
                if (colp[3 * (size_t)Kp + j] != on) {
                    colp[3 * (size_t)Kp + j] = on;
                    flip = true;
                }
            }
            if (flip) {
                LGK_CUDA_TRY(cudaMemcpyAsync(r.colp.as<float>() + 3 * (size_t)Kp, colp.data() + 3 * (size_t)Kp,
                                             (size_t)Kp * 4, cudaMemcpyHostToDevice, st));
                LGK_CUDA_TRY(cudaStreamSynchronize(st));
            }
        }
    }
    cudaFreeHost(hc);
    for (cudaEvent_t e : tev)
        if (e) cudaEventDestroy(e);
    r.colp_h = colp;
    if (rc) return rc;
    if (stream && (rc = flush_checks())) return rc;
    k_objective<<<Kp, 256, 0, st>>>(cx, r.stats.as<double>() + 2 * Kp);
    LGK_LAUNCH_CHECK();
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    return LGK_OK;
}

// ------------------------------------------------------------ group solve

static int fail_status(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

// One iteration of a group (the sequence of iteration_bf16): every tensor-core
// product is one launch over all G solves, and so is every element-wise step
// (member = blockIdx.z), on the group's stream.
static int iteration_group(int G, ResultData* const* R, const IterCtx* cx, cudaStream_t st, int itx) {
    const ResultData& r0 = *R[0];
    const int check_every = r0.cs->prm.check_every;
    const bool test_slot = (itx + 1) % check_every == 0;
    const bool full = r0.refine && (itx == 0 || test_slot);
    const bool first_only = itx == 0 && !test_slot;
    const bool pdl = true;
    const int steps = r0.refine_steps;
    int mx = 1, kx = 1;
    for (int g = 0; g < G; ++g) {
        mx = std::max(mx, R[g]->cs->m_pad / 256);
        kx = std::max(kx, R[g]->Kp);
    }
    const dim3 gm(mx, kx, G);
    // the members' arguments of one element-wise step
    auto ew = [&](auto fill) {
        EwGroup P;
        memset(&P, 0, sizeof(P));
        P.G = G;
        for (int g = 0; g < G; ++g) {
            P.m[g].cx = cx[g];
            fill(*R[g], P.m[g]);
        }
        return P;
    };
    int rc;
    if (full && (rc = tc_group_gemm1_lo(G, R, st, pdl && itx > 0, first_only))) return rc;
    if ((rc = tc_group_gemm1(G, R, st, pdl && (itx > 0 || full)))) return rc;
    {
        EwGroup P = ew([&](ResultData& r, EwMember& m) {
            m.src = plan_src(r, r.plan1);
            m.p0 = r.rhs.p;
            m.f1 = steps ? r.rhs32.as<float>() : nullptr;
        });
        LGK_CUDA_TRY(launch_k(k_reduce_rhs_g, gm, dim3(64), 0, st, pdl, P));
        LGK_LAUNCH_CHECK();
    }
    if ((rc = tc_group_solve(G, R, st, pdl))) return rc;
    auto solve_args = [&](ResultData& r, EwMember& m) {
        m.src = plan_src(r, r.plan_s);
        m.p0 = r.V.p;
        m.f1 = steps ? r.rv.as<float>() : nullptr;
        m.b2 = steps ? r.V3.as<__nv_bfloat16>() : nullptr;
    };
    {
        EwGroup P = ew(solve_args);
        if (steps == 0) LGK_CUDA_TRY(launch_k(k_reduce_solve_g<RS_PLAIN>, gm, dim3(64), 0, st, pdl, P));
        else LGK_CUDA_TRY(launch_k(k_reduce_solve_g<RS_FIRST>, gm, dim3(64), 0, st, pdl, P));
        LGK_LAUNCH_CHECK();
    }
    for (int step = 1; step <= steps; ++step) {
        if ((rc = tc_group_sv(G, R, st, pdl))) return rc;
        {
            EwGroup P = ew([&](ResultData& r, EwMember& m) {
                m.src = plan_src(r, r.plan_s);
                m.p0 = r.rhs.p;
                m.f1 = r.rhs32.as<float>();
            });
            LGK_CUDA_TRY(launch_k(k_reduce_err_g, gm, dim3(64), 0, st, pdl, P));
            LGK_LAUNCH_CHECK();
        }
        if ((rc = tc_group_solve(G, R, st, pdl))) return rc;
        EwGroup P = ew(solve_args);
        if (step < steps) LGK_CUDA_TRY(launch_k(k_reduce_solve_g<RS_ACCUM>, gm, dim3(64), 0, st, pdl, P));
        else LGK_CUDA_TRY(launch_k(k_reduce_solve_g<RS_FINAL>, gm, dim3(64), 0, st, pdl, P));
        LGK_LAUNCH_CHECK();
    }
    if (full && (rc = tc_group_gemm2_lo(G, R, st, pdl, first_only))) return rc;
    if ((rc = tc_group_gemm2(G, R, st, pdl))) return rc;
    {
        EwGroup P = ew([&](ResultData&, EwMember&) {});
        LGK_CUDA_TRY(launch_k(k_finalize_g, dim3(kx, 1, G), dim3(128), 0, st, pdl, P));
        LGK_LAUNCH_CHECK();
    }
    return LGK_OK;
}

int run_group(int G, ResultData* const* R) {
    if (G < 1 || G > 4) return fail_status(LGK_EINVAL, "a group holds 1 to 4 solves");
    const ResultData& r0 = *R[0];
    const CaseData& c0 = *r0.cs;
    for (int g = 0; g < G; ++g) {
        const ResultData& r = *R[g];
        const CaseData& cs = *r.cs;
        if (cs.prm.precision == LGK_PREC_FP32)
            return fail_status(LGK_EINVAL, "group solves run the BF16 forms only");
        if (cs.device != c0.device) return fail_status(LGK_EINVAL, "a group's cases must share one device");
        if (cs.na != c0.na || r.refine != r0.refine || r.refine_steps != r0.refine_steps ||
            cs.prm.check_every != c0.prm.check_every || r.mask_words)
            return fail_status(LGK_EINVAL, "a group's solves must share the iteration form (BF16 terms, lagged "
                                           "low term, solve refinement, residual-test spacing)");
    }
    int rc;
    // one tile height per GEMM for all: 256-row tiles only if every solve can
    // take them
    bool all_wide = true, all_wide2 = true;
    for (int g = 0; g < G; ++g) {
        all_wide = all_wide && R[g]->wide;
        all_wide2 = all_wide2 && R[g]->wide2;
    }
    for (int g = 0; g < G; ++g)
        if (R[g]->wide != all_wide || R[g]->wide2 != all_wide2) {
            R[g]->force_wide = all_wide ? 1 : 0;
            R[g]->force_wide2 = all_wide2 ? 1 : 0;
            if ((rc = tc_prepare(*R[g]))) return rc;
        }
    cudaStream_t st = c0.stream;
    const int per_graph = std::max(1, std::min(r0.max_iter, 5 * c0.prm.check_every));
    std::vector<IterCtx> cx(G);
    for (int g = 0; g < G; ++g) cx[g] = make_ctx(*R[g]);
    // the group's graph of per_graph iterations (captured again when the
    // group changes its iteration form)
    cudaGraphExec_t exec = nullptr;
    struct ExecGuard {
        cudaGraphExec_t* e;
        ~ExecGuard() { if (*e) cudaGraphExecDestroy(*e); }
    } guard{&exec};
    size_t n_nodes = 0;
    auto capture = [&]() -> int {
        cudaGraph_t graph = nullptr;
        LGK_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int it = 0; it < per_graph; ++it) {
            const int rc2 = iteration_group(G, R, cx.data(), st, it);
            if (rc2) {
                cudaStreamEndCapture(st, &graph);
                if (graph) cudaGraphDestroy(graph);
                return rc2;
            }
        }
        LGK_CUDA_TRY(cudaStreamEndCapture(st, &graph));
        size_t n_all = 0;
        n_nodes = 0;
        if (cudaGraphGetNodes(graph, nullptr, &n_all) == cudaSuccess && n_all) {
            std::vector<cudaGraphNode_t> nodes(n_all);
            if (cudaGraphGetNodes(graph, nodes.data(), &n_all) == cudaSuccess)
                for (auto nd : nodes) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++n_nodes;
                }
        }
        count_launch(-(long long)n_nodes);
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess)
            return fail_status(LGK_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
        return LGK_OK;
    };
    if ((rc = capture())) return rc;
    Control* hc = nullptr;
    LGK_CUDA_TRY(cudaMallocHost(&hc, sizeof(Control) * G));
    struct HostGuard {
        Control* p;
        ~HostGuard() { if (p) cudaFreeHost(p); }
    } hguard{hc};
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t le = cudaGraphLaunch(exec, st);
        if (le != cudaSuccess) return fail_status(LGK_ECUDA, cudaGetErrorString(le));
        count_launch((long long)n_nodes);
        for (int g = 0; g < G; ++g)
            LGK_CUDA_TRY(cudaMemcpyAsync(hc + g, R[g]->ctrl.p, sizeof(Control), cudaMemcpyDeviceToHost, st));
        for (;;) {
            cudaError_t q = cudaStreamQuery(st);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) return fail_status(LGK_ECUDA, cudaGetErrorString(q));
            auto el = std::chrono::steady_clock::now() - t0;
            if (std::chrono::duration_cast<std::chrono::milliseconds>(el).count() > c0.prm.timeout_ms)
                return fail_status(LGK_ETIMEOUT, "group solve exceeded timeout_ms");
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        bool any = false;
        int age = 0;             // iterations of the oldest running member
        for (int g = 0; g < G; ++g) {
            if (hc[g].err)
                return fail_status(LGK_ECUDA, "device error flag " + std::to_string(hc[g].err) +
                                                  " raised during the group solve (case " + std::to_string(g) + ")");
            any = any || hc[g].n_active != 0;
            if (hc[g].n_active) age = std::max(age, hc[g].iter);
        }
        if (!any) break;
        if (R[0]->refine && c0.prm.lo_refresh_iters > 0 && age >= c0.prm.lo_refresh_iters) {
            // a member still running this long: as a solo solve does, the
            // group continues with the literal iteration (every term every
            // step; 128-row tiles) from the current state
            cudaGraphExecDestroy(exec);
            exec = nullptr;
            for (int g = 0; g < G; ++g) {
                R[g]->refine = false;
                R[g]->force_wide = R[g]->force_wide2 = -1;
                if ((rc = tc_prepare(*R[g]))) return rc;
                cx[g] = make_ctx(*R[g]);
            }
            if ((rc = capture())) return rc;
        }
    }
    for (int g = 0; g < G; ++g) {
        ResultData& r = *R[g];
        k_objective<<<r.Kp, 256, 0, st>>>(cx[g], r.stats.as<double>() + 2 * r.Kp);
        LGK_LAUNCH_CHECK();
    }
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    return LGK_OK;
}

// Sector times t = D_r rho max(q2 - b, 0) on the beam rows, FP64, K x B, into
// caller-provided device memory (the allocation-free dose entry point).
__global__ void k_times_into(IterCtx cx, int K, double* t) {
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= cx.n_beams || j >= K) return;
    double q = cx.q2[(size_t)j * cx.m_pad + i];
    t[(size_t)j * cx.n_beams + i] = cx.Dr[i] * (double)cx.rho[j] * fmax(q, 0.0);
}

int times_into(const ResultData& r, double* t_dev) {
    ResultData& rr = const_cast<ResultData&>(r);
    CaseData& cs = *rr.cs;
    IterCtx cx = make_ctx(rr);
    dim3 g((cs.n_beams + 255) / 256, r.K);
    k_times_into<<<g, 256, 0, cs.stream>>>(cx, r.K, t_dev);
    LGK_LAUNCH_CHECK();
    return LGK_OK;
}

// Metric counts of plan j over the evaluation points: [0] covered target
// points, [1] points >= min prescription, [2] points >= D/2, [3] points >= D
// (D the common prescription), [4] target points.  Integer atomics: the
// counts do not depend on the order of the additions.
__global__ void k_metric_counts(const double* __restrict__ dose, const int* __restrict__ label,
                                const double* __restrict__ d_presc, double d_min, double d_ref,
                                int n_eval, unsigned long long* counts) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    unsigned c[5] = {0, 0, 0, 0, 0};
    if (e < n_eval) {
        const double d = dose[(size_t)j * n_eval + e];
        const int lab = label[e];
        c[0] = lab >= 0 && d >= d_presc[lab];
        c[1] = d >= d_min;
        c[2] = d >= 0.5 * d_ref;
        c[3] = d >= d_ref;
        c[4] = lab >= 0;
    }
    __shared__ unsigned red[5][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        unsigned v = c[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        unsigned long long s = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[threadIdx.x][i];
        atomicAdd(&counts[(size_t)j * 5 + threadIdx.x], s);
    }
}

// Beam-on time of plan j (Sec. 3.B): per isocenter the longest sector, its
// three collimator times summed; summed over isocenters in a fixed order.
__global__ void k_beam_on_time(const double* __restrict__ t, int n_iso, double* bot) {
    const int j = blockIdx.x;
    const double* tj = t + (size_t)j * 24 * n_iso;
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n_iso; i += blockDim.x) {
        double mx = 0.0;
        for (int sct = 0; sct < 8; ++sct) {
            const double* p = tj + (size_t)(i * 8 + sct) * 3;
            mx = fmax(mx, p[0] + p[1] + p[2]);
        }
        s += mx;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) bot[j] = red[0];
}

int fetch_metrics(const ResultData& r, const double* phi_eval, int n_eval, const int* label,
                  double* coverage, double* selectivity, double* gi, double* bot) {
    ResultData& rr = const_cast<ResultData&>(r);
    CaseData& cs = *rr.cs;
    cudaStream_t st = cs.stream;
    const int B = cs.n_beams, K = r.K;
    DevBuf td, pd, dd, ld, presc, cnt, botd;
    int rc;
    if ((rc = td.alloc((size_t)K * B * 8)) || (rc = pd.alloc((size_t)n_eval * B * 8)) ||
        (rc = dd.alloc((size_t)K * n_eval * 8)) || (rc = ld.alloc((size_t)n_eval * 4)) ||
        (rc = presc.alloc((size_t)cs.n_targets * 8)) || (rc = cnt.alloc((size_t)K * 5 * 8)) ||
        (rc = botd.alloc((size_t)K * 8)))
        return rc;
    LGK_CUDA_TRY(cudaMemcpyAsync(pd.p, phi_eval, pd.bytes, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(ld.p, label, ld.bytes, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(presc.p, cs.d_presc.data(), presc.bytes, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, cnt.bytes, st));
    if ((rc = times_into(r, td.as<double>()))) return rc;
    if ((rc = dgemm(st, false, true, K, n_eval, B, 1.0, td.as<double>(), B, pd.as<double>(), B, 0.0,
                    dd.as<double>(), n_eval)))
        return rc;
    double d_min = cs.d_presc[0], d_max = cs.d_presc[0];
    for (double d : cs.d_presc) d_min = std::min(d_min, d), d_max = std::max(d_max, d);
    dim3 g((n_eval + 255) / 256, K);
    k_metric_counts<<<g, 256, 0, st>>>(dd.as<double>(), ld.as<int>(), presc.as<double>(), d_min,
                                       cs.d_presc[0], n_eval, cnt.as<unsigned long long>());
    LGK_LAUNCH_CHECK();
    k_beam_on_time<<<K, 256, 0, st>>>(td.as<double>(), cs.n_iso, botd.as<double>());
    LGK_LAUNCH_CHECK();
    std::vector<unsigned long long> c((size_t)K * 5);
    std::vector<double> b(K);
    LGK_CUDA_TRY(cudaMemcpyAsync(c.data(), cnt.p, cnt.bytes, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(b.data(), botd.p, botd.bytes, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    const bool equal = d_min == d_max;
    for (int j = 0; j < K; ++j) {
        const unsigned long long* q = &c[(size_t)j * 5];
        if (coverage) coverage[j] = (double)q[0] / (double)std::max(q[4], 1ull);
        if (selectivity) selectivity[j] = (double)q[0] / (double)std::max(q[1], 1ull);
        if (gi) gi[j] = equal ? (double)q[2] / (double)std::max(q[3], 1ull) : NAN;
        if (bot) bot[j] = b[j];
    }
    return LGK_OK;
}

// ------------------------------------------------------------------ fetch

int fetch_times(const ResultData& r, double* t, double* tau) {
    ResultData& rr = const_cast<ResultData&>(r);
    CaseData& cs = *rr.cs;
    cudaStream_t st = cs.stream;
    DevBuf lam;
    int rc;
    if ((rc = lam.alloc((size_t)r.K * cs.m * 8))) return rc;
    IterCtx cx = make_ctx(rr);
    dim3 g((cs.m + 255) / 256, r.K);
    k_lambda<<<g, 256, 0, st>>>(cx, r.K, lam.as<double>());
    LGK_LAUNCH_CHECK();
    std::vector<double> h((size_t)r.K * cs.m);
    LGK_CUDA_TRY(cudaMemcpyAsync(h.data(), lam.p, h.size() * 8, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < r.K; ++j) {
        if (t) std::copy(&h[(size_t)j * cs.m], &h[(size_t)j * cs.m + cs.n_beams], t + (size_t)j * cs.n_beams);
        if (tau)
            std::copy(&h[(size_t)j * cs.m + cs.n_beams], &h[(size_t)j * cs.m + cs.m],
                      tau + (size_t)j * cs.n_iso);
    }
    return LGK_OK;
}

int fetch_doses(const ResultData& r, const double* phi_eval, int n_eval, double* dose) {
    ResultData& rr = const_cast<ResultData&>(r);
    CaseData& cs = *rr.cs;
    cudaStream_t st = cs.stream;
    const int B = cs.n_beams, K = r.K;
    std::vector<double> t((size_t)K * B);
    int rc;
    if ((rc = fetch_times(r, t.data(), nullptr))) return rc;
    DevBuf td, pd, dd;
    if ((rc = td.alloc(t.size() * 8)) || (rc = pd.alloc((size_t)n_eval * B * 8)) ||
        (rc = dd.alloc((size_t)K * n_eval * 8)))
        return rc;
    LGK_CUDA_TRY(cudaMemcpyAsync(td.p, t.data(), td.bytes, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(pd.p, phi_eval, pd.bytes, cudaMemcpyHostToDevice, st));
    // dose[K][E] = t[K][B] . phi_eval[E][B]^T
    if ((rc = dgemm(st, false, true, K, n_eval, B, 1.0, td.as<double>(), B, pd.as<double>(), B, 0.0,
                    dd.as<double>(), n_eval)))
        return rc;
    LGK_CUDA_TRY(cudaMemcpyAsync(dose, dd.p, dd.bytes, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    return LGK_OK;
}

int fetch_stats(const ResultData& r, int* iters, double* obj, double* rel_pri, double* rel_dual,
                uint8_t* converged) {
    CaseData& cs = *r.cs;
    cudaStream_t st = cs.stream;
    const int K = r.K, Kp = r.Kp;
    std::vector<int> it(Kp), act(2 * Kp);
    std::vector<double> stv(3 * Kp);
    LGK_CUDA_TRY(cudaMemcpyAsync(it.data(), r.iters.p, Kp * 4, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(act.data(), r.active.p, 2 * Kp * 4, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(stv.data(), r.stats.p, 3 * Kp * 8, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < K; ++j) {
        if (iters) iters[j] = it[j];
        if (rel_pri) rel_pri[j] = stv[j];
        if (rel_dual) rel_dual[j] = stv[Kp + j];
        if (obj) obj[j] = stv[2 * Kp + j];
        if (converged) converged[j] = (uint8_t)act[Kp + j];
    }
    return LGK_OK;
}

int fetch_state(const ResultData& r, double* q1, double* q2) {
    ResultData& rr = const_cast<ResultData&>(r);
    CaseData& cs = *rr.cs;
    cudaStream_t st = cs.stream;
    DevBuf zd, yd;
    int rc;
    if ((rc = zd.alloc((size_t)r.K * cs.n * 8)) || (rc = yd.alloc((size_t)r.K * cs.m * 8))) return rc;
    IterCtx cx = make_ctx(rr);
    int ne = std::max(cs.n, cs.m);
    dim3 g((ne + 255) / 256, r.K);
    k_state<<<g, 256, 0, st>>>(cx, r.K, zd.as<double>(), yd.as<double>());
    LGK_LAUNCH_CHECK();
    if (q1) LGK_CUDA_TRY(cudaMemcpyAsync(q1, zd.p, zd.bytes, cudaMemcpyDeviceToHost, st));
    if (q2) LGK_CUDA_TRY(cudaMemcpyAsync(q2, yd.p, yd.bytes, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    return LGK_OK;
}

}  // namespace lgk
