// Tensor-core GEMMs of one ADMM iteration on sm_103a: tcgen05.mma (BF16 in,
// FP32 accumulate in TMEM), operands staged by TMA (cp.async.bulk.tensor, 128B
// swizzle, no multicast) through an mbarrier ring, warp-specialised CTA:
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM allocator + MMA issuer (one elected lane)
//   warps 2..9  epilogue: tcgen05.ld of the accumulators, two warps per TMEM
//               lane quarter (one row per thread; the two warps take the two
//               column halves of a 128-row tile, or the two 128-row halves of
//               a 256-row tile)
//
// Output tile: 128 or 256 rows (MT = 1, 2) of the long dimension (m for
// GEMM1 and the solve, n for GEMM2) x N columns (weightings, N <= 256).  The
// kernel is persistent and stream-K scheduled: the (tile, 64-wide k block)
// units of a GEMM are cut into one contiguous run per CTA, so every SM
// streams the same number of operand blocks; a run is split into segments at
// tile boundaries, each segment's partial sum goes to its own slot (up to four
// accumulator sets in TMEM, so the epilogue of one segment overlaps the loads
// and MMAs of the next), and a tile's slots are added in k order
// (deterministic).  Each product A.B is a sum of BF16 x BF16 terms (exact
// products, FP32 sums):
//   GEMM1   A . R1         = A_hi.R1_hi + A_hi.R1_lo + A_lo.R1_hi  (3 terms; with
//                            the lagged low term, A_hi.R1 every iteration and
//                            A_lo.R1_hi on the full ones; the one-term-A form
//                            drops A_lo: 2 terms)
//   solve   S^{-1} . rhs   = G_hi.r_hi + G_hi.r_mid + G_mid.r_hi
//                            + G_hi.r_lo + G_mid.r_mid + G_lo.r_hi (6 terms;
//                            S^{-1} and rhs each split into three BF16 parts,
//                            because S amplifies the rounding of its input)
//   GEMM2   A^T . V        = A_hi^T.V_hi + A_hi^T.V_lo + A_lo^T.V_hi (as GEMM1)
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "iter_ctx.cuh"
#include "lgk_impl.hpp"
#include "tc_ptx.cuh"

namespace lgk {

// term t of an NT-term product: which A part and which B part.
//   NT = 1: A.B (one part each: the lagged low-term products)
//   NT = 2: A.B_hi + A.B_lo
//   NT = 3: A_hi.B_hi + A_hi.B_lo + A_lo.B_hi
//   NT = 5: two parts of A, three of B, all (a, b) with a + b <= 2
//   NT = 6: all (a, b) with a + b <= 2 over three parts each
// (dropped terms are below 2^-16 resp. 2^-24 of the product, relative).
// NT = 5 and 6 share the order (0,0) (0,1) (1,0) (0,2) (1,1) [(2,0)].
__host__ __device__ constexpr int term_a(int NT, int t) {
    return NT <= 2 ? 0 : NT == 3 ? (t == 2 ? 1 : 0)
                               : (t == 0 || t == 1 || t == 3 ? 0 : (t == 2 || t == 4 ? 1 : 2));
}
__host__ __device__ constexpr int term_b(int NT, int t) {
    return NT == 1 ? 0 : NT == 2 ? t : NT == 3 ? (t == 1 ? 1 : 0)
                               : (t == 0 || t == 2 || t == 5 ? 0 : (t == 1 || t == 4 ? 1 : 2));
}


struct TcArgs {
    const int* cta_seg;     // segments of CTA c: [cta_seg[c], cta_seg[c + 1])
    const int* seg;         // 5 ints per segment: row tile, column tile, kb begin, kb end, slot
    const int* tile_begin;  // slots of output tile t: tile_slots[tile_begin[t] .. tile_begin[t + 1])
    const int* tile_slots;
    int* tile_count;        // per output tile: segments finished this launch (reset by the last)
    int row_tiles;
    int n_tile;             // columns per tile (multiple of 16, <= 256)
    int tmem_cols;          // columns of one accumulator (power of two >= n_tile)
    int nbuf;               // accumulators in TMEM (2 or 4; nbuf * tmem_cols <= 512)
    int stages;
    int stage_bytes;
    int out_ld;             // EPI_STORE: rows of the output matrix (m_pad or n_pad)
    int first_only;         // do the work only in the solve's first iteration (else return)
    int keep_a;             // load A with an evict-last L2 policy (S^{-1} kept in L2 across iterations)
    int ncta;               // CTAs with a run in this case's plan (the rest skip the case)
    float* part;            // [slot][n_tile][128] partial sums of tiles split over segments
    void* out;              // EPI_STORE: float [Kp][out_ld];
                            // EPI_Q1: R1 [2][Kp][n_pad] (BF16 terms)
};

// What a finished output tile becomes.  EPI_PARTIAL: every segment stores its
// partial sum in its slot and a separate element-wise kernel adds a tile's
// slots (GEMM1 and the solve: few output tiles, each split over many CTAs,
// so finishing them inside the GEMM would leave the summing to a handful of
// CTAs at the end of the kernel).  Otherwise the CTA that completes a tile
// sums its slots in k order and applies:
//   EPI_Q1     W = A^T V: q1' = P1(q1) - c/rho - W, R1' = 2 P1(q1') - q1' - c/rho
//              as two BF16 terms, residual partials of the n-block (W plus the
//              lagged low-term product lo^T v when iterating with A_hi)
//   EPI_STORE  the product as FP32 [Kp][out_ld] (the lagged low-term products)
enum { EPI_Q1 = 2, EPI_PARTIAL = 3, EPI_STORE = 4 };

constexpr int kThreads = 320;               // 2 producer/MMA warps + 8 epilogue warps
constexpr int kChunk = 8;                   // columns per epilogue step
static_assert(32 % kChunk == 0, "a chunk's columns must share one point-selection word");
constexpr int kABytes = 128 * 64 * 2;       // one 128 x 64 BF16 operand tile

__device__ inline void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// The q1 step (EPI_Q1) in two halves, so the epilogue can load one chunk's
// inputs while it finishes the previous one.
struct Q1In {
    float q[kChunk], u[kChunk], ir[kChunk], c2[kChunk];
    int act[kChunk];
    float c_p;
};

__device__ inline void q1_load(const IterCtx& cx, int row, int j0, Q1In& in) {
    const float* q1p = cx.q1 + (size_t)j0 * cx.n_pad + row;
    const int sl = cx.col_slot[row];
    in.c_p = cx.c_slot[sl];
    // the chunk's 8 columns share one word of the point selection (j0 % 8 == 0)
    const uint32_t sel =
        cx.mask ? __ldg(cx.mask + (size_t)row * cx.mask_words + (j0 >> 5)) >> (j0 & 31) : 0xffu;
    const float* c2p = cx.c2 ? cx.c2 + (size_t)j0 * cx.n_pad + row : nullptr;
#pragma unroll
    for (int c = 0; c < kChunk; ++c) {
        in.q[c] = q1p[(size_t)c * cx.n_pad];
        in.u[c] = ((sel >> c) & 1u) ? __ldg(cx.utab + (j0 + c) * cx.n_slot + sl) : 0.0f;
        in.ir[c] = __ldg(cx.inv_rho + j0 + c);
        in.act[c] = cx.active[j0 + c];
        in.c2[c] = c2p ? __ldcg(c2p + (size_t)c * cx.n_pad) : 0.0f;
    }
}

// W = v (+ the lagged lo^T v): q1' = P1(q1) - c/rho - W, R1' as two BF16 terms.
__device__ inline void q1_finish(const IterCtx& cx, const TcArgs& a, int row, int j0, const float v[kChunk],
                                 const Q1In& in, float res[kChunk][5]) {
    const size_t plane = (size_t)cx.Kp * cx.n_pad;
    float* q1p = cx.q1 + (size_t)j0 * cx.n_pad + row;
    __nv_bfloat16* d = static_cast<__nv_bfloat16*>(a.out) + (size_t)j0 * cx.n_pad + row;
#pragma unroll
    for (int c = 0; c < kChunk; ++c) {
        Q1Update qq = q1_update(in.q[c], v[c] + in.c2[c], in.u[c], in.c_p * in.ir[c]);
        const size_t o = (size_t)c * cx.n_pad;
        if (in.act[c]) q1p[o] = qq.qn;
        __nv_bfloat16 hi, lo;
        split_bf16(qq.r1, hi, lo);
        d[o] = hi;
        d[plane + o] = lo;
#pragma unroll
        for (int k = 0; k < 5; ++k) res[c][k] = qq.res[k];
    }
}

// Apply the element-wise step to kChunk columns [j0, j0 + kChunk) of row `row`,
// accumulating the 5 residual terms per column (block-reduced by the caller).
// Only 8 warps per SM run this, so every input of the chunk's columns is loaded
// before anything is computed or stored: the loads are then in flight
// together instead of one dependent round trip per column.
template <int EPI>
__device__ inline void epi_op(const IterCtx& cx, const TcArgs& a, int row, int j0, const float v[kChunk],
                              float res[kChunk][5]) {
    if (EPI == EPI_STORE) {
        float* o = static_cast<float*>(a.out) + (size_t)j0 * a.out_ld + row;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) o[(size_t)c * a.out_ld] = v[c];
    } else {
        Q1In in;
        q1_load(cx, row, j0, in);
        q1_finish(cx, a, row, j0, v, in, res);
    }
}

// Reduce the residual terms of kChunk columns over 128 rows (the 4 warps of
// group `hf`: one column half of a 128-row tile, or one 128-row half of a
// 256-row tile) and store them as that 128-row block's partial for those
// columns.  Both groups call it the same number of times (barriers).
__device__ inline void epi_resid(float res[kChunk][5], float* red, double* dst, int lane, int ew, int hf,
                                 int et) {
#pragma unroll
    for (int c = 0; c < kChunk; ++c)
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float v = res[c][k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[((hf * 4 + ew) * kChunk + c) * 5 + k] = v;
        }
    epi_bar();
    const int e = et & 127;
    if (e < kChunk * 5) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < 4; ++w) s += (double)red[(hf * 4 + w) * kChunk * 5 + e];
        dst[e] = s;
    }
    epi_bar();
}

// The A tiles of one stage (k block kx, output rows row0 ..): NA terms x MT
// sub-tiles of 128 rows; an MN-major tile is two 64-row boxes.
template <int NA, int NT, bool A_MN, int EPI, int MT>
__device__ inline void load_a_stage(const CUtensorMap* tmA, uint32_t st, uint32_t full, int row0, int kx,
                                    uint64_t pol_a, bool keep) {
    if (A_MN) {
#pragma unroll
        for (int p = 0; p < NA; ++p)
#pragma unroll
            for (int h = 0; h < MT; ++h) {
                const uint32_t dst = st + (p * MT + h) * kABytes;
                tma_load_3d_hint(dst, tmA, row0 + h * 128, kx, p, full, pol_a);
                tma_load_3d_hint(dst + kABytes / 2, tmA, row0 + h * 128 + 64, kx, p, full, pol_a);
            }
    } else if (EPI == EPI_PARTIAL && NT == 6) {
        // the solve: S^{-1} is re-read every iteration: default policy, or
        // evict-last when a persisting L2 carve-out holds it (keep_a)
        if (keep) {
#pragma unroll
            for (int p = 0; p < NA; ++p) tma_load_3d_hint(st + p * kABytes, tmA, kx, row0, p, full, pol_a);
        } else {
#pragma unroll
            for (int p = 0; p < NA; ++p) tma_load_3d(st + p * kABytes, tmA, kx, row0, p, full);
        }
    } else {
#pragma unroll
        for (int p = 0; p < NA; ++p)
#pragma unroll
            for (int h = 0; h < MT; ++h)
                tma_load_3d_hint(st + (p * MT + h) * kABytes, tmA, kx, row0 + h * 128, p, full, pol_a);
    }
}

// Up to kMaxGroup cases in one launch (a co-scheduled group solve, Sec. 2.B's
// K columns generalised to several matrices): every CTA runs its stream-K run
// of case 0's units, then its run of case 1's, and so on, through one
// continuous TMA / MMA / epilogue pipeline (no drain between cases).  Each
// case's plan is cut into its own equal runs, so the group stays balanced and
// every case's tiles are summed exactly as in a launch of that case alone.
constexpr int kMaxGroup = 4;
struct TcGroup {
    CUtensorMap tmA[kMaxGroup];
    CUtensorMap tmB[kMaxGroup];
    TcArgs a[kMaxGroup];      // stages, stage_bytes, tmem_cols, nbuf, first_only, keep_a: launch-wide (a[0])
    IterCtx cx[kMaxGroup];
    int G;
};
static_assert(sizeof(TcGroup) <= 4096, "kernel parameters of a group launch exceed 4 KB");

// MT: 128-row sub-tiles per output tile.  MT = 2 puts two accumulators side by
// side (256 rows) on one B tile: half the B traffic per A byte, and twice the
// A bytes per pipeline stage, so more of A is in flight per SM (the one-term-A
// GEMMs are otherwise limited by how much of A the stage ring holds).
template <int NA, int NB, int NT, bool A_MN, int EPI, int MT>
__global__ void __launch_bounds__(kThreads, 1) k_tc_gemm(const __grid_constant__ TcGroup P) {
    pdl_trigger();
    const TcArgs& a0 = P.a[0];
    const int G = P.G;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int S = a0.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * a0.stage_bytes);
    // bars: [0, S) stage full, [S, 2S) stage empty, 2S + b accumulator b full,
    // 2S + 4 + b accumulator b drained (b < nbuf <= 4)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 8);
    int* sh_last = reinterpret_cast<int*>(bars + 2 * S + 8) + 1;
    int* sh_run = reinterpret_cast<int*>(bars + 2 * S + 9);         // bit g: case g has work
    int* sh_pre = sh_run + 1;                                       // stages prefetched for case 0
    float* red = reinterpret_cast<float*>(bars + 2 * S + 10);       // [8 warps][kChunk][5]
    const int NBUF = a0.nbuf;
    const int TC = a0.tmem_cols;                                    // columns of one accumulator

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * S + 4; ++s) mbar_init(smem_u32(&bars[s]), 1);
        for (int b = 0; b < 4; ++b) mbar_init(smem_u32(&bars[2 * S + 4 + b]), 8);   // one per epilogue warp
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), NBUF * MT * TC);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // The A operand (the case matrix's BF16 terms, or S^{-1}) is written at
    // set-up and by no kernel of the iteration, so the first stages' A tiles
    // are loaded before the wait on the previous kernel and arrive during its
    // tail.  Their bytes are added to the stage's full barrier as a pending
    // transaction without an arrival: the stage cannot complete before the
    // arrival that comes with its B tile, after the wait.  (Not for launches
    // that work only in the solve's first iteration: they mostly do nothing;
    // not for groups.)
    const uint32_t a_bytes = (uint32_t)(NA * MT * kABytes);
    int pre = 0;
    if (G == 1 && !a0.first_only && warp == 0 && lane == 0 && (int)blockIdx.x < a0.ncta) {
        const int s0 = a0.cta_seg[blockIdx.x], s1 = a0.cta_seg[blockIdx.x + 1];
        prefetch_tmap(&P.tmA[0]);
        prefetch_tmap(&P.tmB[0]);
        const uint64_t pol_a = a0.keep_a ? policy_evict_last() : policy_evict_first();
        for (int sg = s0; sg < s1 && pre < S; ++sg) {
            const int* g = a0.seg + 5 * sg;
            for (int kb = g[2]; kb < g[3] && pre < S; ++kb, ++pre) {
                const uint32_t full = smem_u32(&bars[pre]);
                mbar_expect_tx_only(full, a_bytes);
                load_a_stage<NA, NT, A_MN, EPI, MT>(&P.tmA[0], smem_u32(smem + (size_t)pre * a0.stage_bytes), full,
                                                    g[0] * 128 * MT, kb * 64, pol_a, a0.keep_a != 0);
            }
        }
    }
    // set-up done; from here on the previous kernel's output is read
    pdl_wait();
    if (threadIdx.x == 0) {
        int m = 0;
        for (int g = 0; g < G; ++g) {
            const Control* c = P.cx[g].ctrl;
            if ((int)blockIdx.x < P.a[g].ncta && c->n_active != 0 && c->err == 0 &&
                (!a0.first_only || c->iter == 0))
                m |= 1 << g;
        }
        *sh_run = m;
        *sh_pre = pre;                                  // thread 0 is the producer
    }
    __syncthreads();
    const int runmask = *sh_run;
    // stages prefetched for a solve that has stopped (or has an error
    // pending): the producer lets them land and both pipelines start after them
    const int skip = (runmask & 1) ? 0 : *sh_pre;

    if (warp == 0 && lane == 0) {
        int* err = &P.cx[0].ctrl->err;
        for (int s = 0; s < skip; ++s) {
            mbar_arrive(smem_u32(&bars[s]));
            mbar_wait(smem_u32(&bars[s]), 0u, err);
        }
        // ---------------- TMA producer: one continuous stream of k blocks
        bool ok = true;
        int it = skip;
        // A streams through once per launch; the B operand, S^{-1} and the
        // epilogue's state should outlive it in L2
        const uint64_t pol_a = a0.keep_a ? policy_evict_last() : policy_evict_first();
#pragma unroll
        for (int gi = 0; gi < kMaxGroup; ++gi) {
            if (gi >= G || !ok) break;
            if (!((runmask >> gi) & 1)) continue;
            const TcArgs& a = P.a[gi];
            err = &P.cx[gi].ctrl->err;
            const int s0 = a.cta_seg[blockIdx.x], s1 = a.cta_seg[blockIdx.x + 1];
            const int b_bytes = a.n_tile * 128;
            for (int sg = s0; sg < s1 && ok; ++sg) {
                const int* g = a.seg + 5 * sg;
                const int row0 = g[0] * 128 * MT, col0 = g[1] * a.n_tile;
                for (int kb = g[2]; kb < g[3] && ok; ++kb, ++it) {
                    const int s = it % S;
                    const uint32_t ph = (uint32_t)(it / S) & 1u;
                    const uint32_t full = smem_u32(&bars[s]);
                    const uint32_t st = smem_u32(smem + (size_t)s * a0.stage_bytes);
                    const int kx = kb * 64;
                    if (it < pre) {
                        // A already in flight (prefetched): the arrival and the B bytes
                        mbar_expect_tx(full, a_bytes + (uint32_t)(NB * b_bytes) - a_bytes);
                    } else {
                        ok = mbar_wait(smem_u32(&bars[S + s]), ph ^ 1u, err);
                        if (!ok) break;
                        mbar_expect_tx(full, a_bytes + (uint32_t)(NB * b_bytes));
                        load_a_stage<NA, NT, A_MN, EPI, MT>(&P.tmA[gi], st, full, row0, kx, pol_a, a0.keep_a != 0);
                    }
                    const uint32_t sb = st + a_bytes;
#pragma unroll
                    for (int p = 0; p < NB; ++p) tma_load_3d(sb + p * b_bytes, &P.tmB[gi], kx, col0, p, full);
                }
            }
        }
        // drain: wait (bounded) for the copies of the last issued stages
        for (int j = max(0, it - S); j < it && ok; ++j)
            ok = mbar_wait(smem_u32(&bars[j % S]), (uint32_t)(j / S) & 1u, err);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        bool ok = true;
        int it = skip, u = 0;
        for (int s = 0; s < skip; ++s) mbar_arrive(smem_u32(&bars[S + s]));   // skipped stages are free
#pragma unroll
        for (int gi = 0; gi < kMaxGroup; ++gi) {
            if (gi >= G) break;
            if (!((runmask >> gi) & 1)) continue;
            const TcArgs& a = P.a[gi];
            int* err = &P.cx[gi].ctrl->err;
            const int s0 = a.cta_seg[blockIdx.x], s1 = a.cta_seg[blockIdx.x + 1];
            const int b_bytes = a.n_tile * 128;
            const uint32_t idesc = instr_desc(a.n_tile, A_MN);
            for (int sg = s0; sg < s1; ++sg, ++u) {
                const int* g = a.seg + 5 * sg;
                const int b = u % NBUF;
                if (ok) ok = mbar_wait(smem_u32(&bars[2 * S + 4 + b]), (uint32_t)((u / NBUF) & 1) ^ 1u, err);
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * MT * TC);
                for (int kb = g[2]; kb < g[3]; ++kb, ++it) {
                    const int s = it % S;
                    const uint32_t ph = (uint32_t)(it / S) & 1u;
                    if (ok) ok = mbar_wait(smem_u32(&bars[s]), ph, err);
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + (size_t)s * a0.stage_bytes);
                    const uint32_t sb = st + NA * MT * kABytes;
                    if (ok) {
#pragma unroll
                        for (int t = 0; t < NT; ++t) {
                            const uint32_t sbt = sb + term_b(NT, t) * b_bytes;
#pragma unroll
                            for (int h = 0; h < MT; ++h) {
                                const uint32_t sa = st + (term_a(NT, t) * MT + h) * kABytes;
#pragma unroll
                                for (int ks = 0; ks < 4; ++ks) {
                                    uint64_t ad = A_MN ? smem_desc(sa + ks * 2048, kABytes / 2, 1024)
                                                       : smem_desc(sa + ks * 32, 16, 1024);
                                    uint64_t bd = smem_desc(sbt + ks * 32, 16, 1024);
                                    tc_mma(d + (uint32_t)(h * TC), ad, bd, idesc,
                                           (kb > g[2] || t > 0 || ks > 0) ? 1u : 0u);
                                }
                            }
                        }
                    }
                    tc_commit(smem_u32(&bars[S + s]));      // frees the stage when its MMAs finish
                }
                tc_commit(smem_u32(&bars[2 * S + b]));      // accumulator b complete
            }
        }
    } else if (warp >= 2) {
        // ---------------- epilogue (8 warps)
        const int ew = warp & 3;                        // TMEM lane quarter of this warp
        const int hf = (warp - 2) >> 2;                 // MT = 1: column half; MT = 2: row half
        const int et = threadIdx.x - 64;                // 0..255
        const int r = ew * 32 + lane;                   // row within the 128-row sub-tile
        const int hrow = MT == 2 ? hf : 0;              // this warp's 128-row sub-tile
        bool ok = true;
        int u = 0;
#pragma unroll
        for (int gi = 0; gi < kMaxGroup; ++gi) {
            if (gi >= G) break;
            if (!((runmask >> gi) & 1)) continue;
            const TcArgs& a = P.a[gi];
            const IterCtx& cx = P.cx[gi];
            int* err = &cx.ctrl->err;
            const int s0 = a.cta_seg[blockIdx.x], s1 = a.cta_seg[blockIdx.x + 1];
            const int half = a.n_tile / 2;              // multiple of kChunk
            const int cbeg = MT == 2 ? 0 : hf * half, cend = MT == 2 ? a.n_tile : cbeg + half;
            const bool check = EPI == EPI_Q1 && is_check_iter(cx.ctrl, cx.check_every, cx.tol);
            for (int sg = s0; sg < s1; ++sg, ++u) {
                const int b = u % NBUF;
                const int* g = a.seg + 5 * sg;
                const int rt = g[0], ct = g[1], slot = g[4];
                const int tile = ct * a.row_tiles + rt;
                const int sb = a.tile_begin[tile], se = a.tile_begin[tile + 1];
                const int row = (rt * MT + hrow) * 128 + r, col0 = ct * a.n_tile;
                double* rdst = cx.resid +
                               ((size_t)(rt * MT + hrow) * cx.Kp + col0) * 5;
                // a whole tile of the q1 step: the state of its first two
                // chunks is loaded before the wait for the accumulator, so the
                // loads are in flight while the tile's k loop still runs (the
                // epilogue of a CTA's last tile is otherwise exposed).  Only
                // this epilogue writes these rows of q1 in this launch.
                Q1In inA, inB;
                if (EPI == EPI_Q1 && se - sb == 1) {
                    q1_load(cx, row, col0 + cbeg, inA);
                    if (cbeg + kChunk < cend) q1_load(cx, row, col0 + cbeg + kChunk, inB);
                }
                if (ok) ok = mbar_wait(smem_u32(&bars[2 * S + b]), (uint32_t)((u / NBUF) & 1), err);
                tc_fence_after();
                const uint32_t base =
                    tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)((b * MT + hrow) * TC);
                if (EPI == EPI_PARTIAL || se - sb > 1) {
                    // store this segment's partial sum in its slot ([slot][MT][n_tile][128])
                    float* own = a.part + ((size_t)slot * MT + hrow) * a.n_tile * 128 + r;
                    for (int c0 = cbeg; c0 < cend; c0 += kChunk) {
                        float v[kChunk];
                        tmem_ld8(base + (uint32_t)c0, v);
#pragma unroll
                        for (int c = 0; c < kChunk; ++c) own[(size_t)(c0 + c) * 128] = ok ? v[c] : 0.f;
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&bars[2 * S + 4 + b]));
                    if (EPI != EPI_PARTIAL) {
                        // the CTA completing the tile sums its slots in k order
                        __threadfence();
                        epi_bar();
                        if (et == 0) *sh_last = atomicAdd(&a.tile_count[tile], 1) == se - sb - 1;
                        epi_bar();
                        if (*sh_last) {
                            __threadfence();
                            for (int c0 = cbeg; c0 < cend; c0 += kChunk) {
                                float v[kChunk], res[kChunk][5];
#pragma unroll
                                for (int c = 0; c < kChunk; ++c) v[c] = 0.f;
                                for (int k = sb; k < se; ++k) {
                                    const float* ps =
                                        a.part + ((size_t)a.tile_slots[k] * MT + hrow) * a.n_tile * 128 + r;
#pragma unroll
                                    for (int c = 0; c < kChunk; ++c) v[c] += __ldcg(ps + (size_t)(c0 + c) * 128);
                                }
                                epi_op<EPI>(cx, a, row, col0 + c0, v, res);
                                if (check) epi_resid(res, red, rdst + c0 * 5, lane, ew, hf, et);
                            }
                            if (et == 0) a.tile_count[tile] = 0;
                        }
                        epi_bar();
                    }
                } else if (EPI == EPI_Q1) {
                    // the whole k range of the tile is in this accumulator; two
                    // chunks' inputs are in flight while one is finished (two
                    // named buffers, unrolled by two, so both stay in registers)
                    float vA[kChunk], vB[kChunk], res[kChunk][5];
                    tmem_ld8(base + (uint32_t)cbeg, vA);
                    for (int c0 = cbeg; c0 < cend; c0 += 2 * kChunk) {
                        const bool moreB = c0 + kChunk < cend;
                        if (!ok)
                            for (int c = 0; c < kChunk; ++c) vA[c] = 0.f;
                        q1_finish(cx, a, row, col0 + c0, vA, inA, res);
                        if (check) epi_resid(res, red, rdst + c0 * 5, lane, ew, hf, et);
                        if (!moreB) break;
                        tmem_ld8(base + (uint32_t)(c0 + kChunk), vB);
                        const bool moreA = c0 + 2 * kChunk < cend;
                        if (moreA) q1_load(cx, row, col0 + c0 + 2 * kChunk, inA);
                        if (!ok)
                            for (int c = 0; c < kChunk; ++c) vB[c] = 0.f;
                        q1_finish(cx, a, row, col0 + c0 + kChunk, vB, inB, res);
                        if (check) epi_resid(res, red, rdst + (c0 + kChunk) * 5, lane, ew, hf, et);
                        if (c0 + 3 * kChunk < cend) q1_load(cx, row, col0 + c0 + 3 * kChunk, inB);
                        if (moreA) tmem_ld8(base + (uint32_t)(c0 + 2 * kChunk), vA);
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&bars[2 * S + 4 + b]));
                } else {
                    // the whole k range of the tile is in this accumulator
                    for (int c0 = cbeg; c0 < cend; c0 += kChunk) {
                        float v[kChunk], res[kChunk][5];
                        tmem_ld8(base + (uint32_t)c0, v);
                        if (!ok)
                            for (int c = 0; c < kChunk; ++c) v[c] = 0.f;
                        epi_op<EPI>(cx, a, row, col0 + c0, v, res);
                        if (check) epi_resid(res, red, rdst + c0 * 5, lane, ew, hf, et);
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&bars[2 * S + 4 + b]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, NBUF * MT * TC);
    }
}

// ------------------------------------------------------------- host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    // thread-safe one-time lookup (the serving workers create maps concurrently)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }();
    return fn;
}

// BF16 tensor map of `parts` stacked [rows][cols] matrices, box 64 x box_rows.
static int make_map(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint64_t parts,
                    uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled entry point unavailable");
        return LGK_ECUDA;
    }
    if (((uintptr_t)base & 15) || (cols * 2) % 16) {
        set_error("tensor map: base or row stride not 16-byte aligned");
        return LGK_EINVAL;
    }
    cuuint64_t dims[3] = {cols, rows, parts};
    cuuint64_t strides[2] = {cols * 2, cols * rows * 2};
    cuuint32_t box[3] = {64, box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box,
                    es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
        return LGK_ECUDA;
    }
    return LGK_OK;
}

int make_tma_map(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint64_t parts,
                 uint32_t box_rows) {
    return make_map(m, base, cols, rows, parts, box_rows);
}

static constexpr int kSmemLimit = 232448;    // 227 KB opt-in per block

static int smem_extra() { return 1024 + 8 * (2 * 8 + 8) + 32 + 8 * kChunk * 5 * 4; }

int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
        return v;
    }();
    return n;
}

// Stream-K plan: the units (column tile, row tile, k block), in that order,
// cut into `grid` contiguous runs of equal length (+-1), each run split into
// segments at tile boundaries.  Depends only on the GEMM's shape.
int build_plan(GemmPlan& P, int rows, int col_tiles, int kb_total, int n_tile, bool split_first, int mt,
               int max_seg) {
    const long long T = (long long)rows * col_tiles;
    const long long U = T * kb_total;
    const int grid = (int)std::min<long long>(sm_count(), U);
    std::vector<int> cta_seg(grid + 1), seg, tile_begin(rows * col_tiles + 1, 0);
    std::vector<std::vector<int>> per_tile(rows * col_tiles);
    int nseg = 0;
    auto add = [&](long long tile, int kb0, int kb1) {
        int ct = (int)(tile / rows), rt = (int)(tile % rows);
        seg.insert(seg.end(), {rt, ct, kb0, kb1, nseg});
        per_tile[tile].push_back(nseg);
        ++nseg;
    };
    // split_first (a GEMM that finishes its tiles in its own epilogue): every
    // CTA owns floor(T / grid) whole tiles and the remaining tiles' k blocks
    // are shared out evenly; each CTA runs its shared pieces first, so the
    // tiles assembled from several CTAs' partial sums complete early and the
    // last work of every CTA is a whole tile (no partial sums to gather).
    const long long full = split_first ? T / grid : 0;
    const long long t_split0 = full * grid;             // tiles [t_split0, T) are shared
    const long long Us = (T - t_split0) * kb_total;
    for (int c = 0; c < grid; ++c) {
        cta_seg[c] = nseg;
        long long u0 = t_split0 * kb_total + Us * c / grid, u1 = t_split0 * kb_total + Us * (c + 1) / grid;
        while (u0 < u1) {
            long long tile = u0 / kb_total;
            int kb0 = (int)(u0 % kb_total);
            int kb1 = (int)std::min<long long>(kb_total, kb0 + (u1 - u0));
            if (max_seg > 0) kb1 = std::min(kb1, (kb0 / max_seg + 1) * max_seg);   // segments inside aligned chunks
            add(tile, kb0, kb1);
            u0 += kb1 - kb0;
        }
        for (long long f = 0; f < full; ++f) add((long long)c * full + f, 0, kb_total);
    }
    cta_seg[grid] = nseg;
    // number the slots tile by tile, in k order, so a tile's partial sums are
    // contiguous: slot = tile_begin[t] + position of the segment in the tile
    std::vector<int> tile_slots;
    for (size_t t = 0; t < per_tile.size(); ++t) {
        tile_begin[t] = (int)tile_slots.size();
        for (int sid : per_tile[t]) {
            seg[5 * sid + 4] = (int)tile_slots.size();
            tile_slots.push_back((int)tile_slots.size());
        }
    }
    tile_begin[per_tile.size()] = (int)tile_slots.size();
    std::vector<int> all;
    all.insert(all.end(), rows * col_tiles, 0);          // tile_count, zero between launches
    all.insert(all.end(), cta_seg.begin(), cta_seg.end());
    all.insert(all.end(), seg.begin(), seg.end());
    all.insert(all.end(), tile_begin.begin(), tile_begin.end());
    all.insert(all.end(), tile_slots.begin(), tile_slots.end());
    int rc;
    if ((rc = P.buf.alloc(all.size() * 4))) return rc;
    LGK_CUDA_TRY(cudaMemcpy(P.buf.p, all.data(), all.size() * 4, cudaMemcpyHostToDevice));
    int* d0 = P.buf.as<int>();
    P.tile_count = d0;
    const int* d = d0 + rows * col_tiles;
    P.grid = grid;
    P.mt = mt;
    P.nseg = nseg;
    P.rows = rows;
    P.col_tiles = col_tiles;
    P.n_tile = n_tile;
    P.cta_seg = d;
    P.seg = d + grid + 1;
    P.tile_begin = d + grid + 1 + 5 * nseg;
    P.tile_slots = P.tile_begin + rows * col_tiles + 1;
    return LGK_OK;
}

template <int NA, int NB, int NT, bool A_MN, int EPI, int MT = 1>
static int launch_in(const CUtensorMap& mA, const CUtensorMap& mB, const GemmPlan& P, CaseData& cs,
                     const IterCtx& cx, float* part, cudaStream_t st);

// Per-case arguments of one launch from a plan.
static TcArgs plan_args(const GemmPlan& P, float* part, void* out, int out_ld) {
    TcArgs a{};
    a.cta_seg = P.cta_seg;
    a.seg = P.seg;
    a.tile_begin = P.tile_begin;
    a.tile_slots = P.tile_slots;
    a.tile_count = P.tile_count;
    a.row_tiles = P.rows;
    a.n_tile = P.n_tile;
    a.ncta = P.grid;
    a.part = part;
    a.out = out;
    a.out_ld = out_ld;
    return a;
}

// Launch-wide fields (ring stages, accumulators) for the widest case of a
// group, copied into every case's arguments; returns the dynamic shared
// memory size, or 0 with the error set.
template <int NA, int NB, int MT>
static size_t group_layout(TcGroup& g, bool first_only, bool keep_a) {
    int nt = 16;
    for (int i = 0; i < g.G; ++i) nt = std::max(nt, g.a[i].n_tile);
    const int stage_bytes = NA * MT * kABytes + NB * nt * 128;
    const int stages = std::min(8, (kSmemLimit - smem_extra()) / stage_bytes);
    if (stages < 2) {
        set_error("tensor-core GEMM: stage does not fit in shared memory");
        return 0;
    }
    int tc = 32;
    while (tc < nt) tc <<= 1;
    const int nbuf = 4 * MT * tc <= 512 ? 4 : 2;
    if (nbuf * MT * tc > 512) {
        set_error("tensor-core GEMM: accumulators exceed tensor memory");
        return 0;
    }
    for (int i = 0; i < g.G; ++i) {
        g.a[i].stage_bytes = stage_bytes;
        g.a[i].stages = stages;
        g.a[i].tmem_cols = tc;
        g.a[i].nbuf = nbuf;
        g.a[i].first_only = first_only;
        g.a[i].keep_a = keep_a;
    }
    return (size_t)stages * stage_bytes + smem_extra();
}

template <int NA, int NB, int NT, bool A_MN, int EPI, int MT = 1>
static int launch(const CUtensorMap& mA, const CUtensorMap& mB, const GemmPlan& P, ResultData& r,
                  void* out, bool pdl, bool first_only = false, bool keep_a = false) {
    if (P.mt != MT) {
        set_error("tensor-core GEMM: plan built for another tile height");
        return LGK_EINVAL;
    }
    TcGroup g;
    memset(&g, 0, sizeof(g));
    g.G = 1;
    g.tmA[0] = mA;
    g.tmB[0] = mB;
    g.a[0] = plan_args(P, r.part.as<float>(), out, A_MN ? r.cs->n_pad : r.cs->m_pad);
    g.cx[0] = make_ctx_public(r);
    const bool keep = keep_a && r.l2_keep;
    const size_t smem = group_layout<NA, NB, MT>(g, first_only, keep);
    if (!smem) return LGK_EINVAL;
    LGK_CUDA_TRY(launch_k_win(k_tc_gemm<NA, NB, NT, A_MN, EPI, MT>, dim3(P.grid), dim3(kThreads), smem,
                              r.cs->stream, pdl, keep ? &r.l2win : nullptr, g));
    LGK_LAUNCH_CHECK();
    return LGK_OK;
}

// One launch over the G solves of a group (run_group): each solve's own maps,
// plan, partial-sum buffer, output and context, on stream st.
template <int NA, int NB, int NT, bool A_MN, int EPI, int MT>
static int launch_group(int G, ResultData* const* R, const CUtensorMap* const* mA, const CUtensorMap* const* mB,
                        const GemmPlan* const* P, void* const* out, cudaStream_t st, bool pdl, bool first_only) {
    if (G < 1 || G > kMaxGroup) {
        set_error("tensor-core GEMM: group size out of range");
        return LGK_EINVAL;
    }
    TcGroup g;
    memset(&g, 0, sizeof(g));
    g.G = G;
    int grid = 1;
    for (int i = 0; i < G; ++i) {
        if (P[i]->mt != MT) {
            set_error("tensor-core GEMM: plan built for another tile height");
            return LGK_EINVAL;
        }
        g.tmA[i] = *mA[i];
        g.tmB[i] = *mB[i];
        g.a[i] = plan_args(*P[i], R[i]->part.as<float>(), out ? out[i] : nullptr,
                           A_MN ? R[i]->cs->n_pad : R[i]->cs->m_pad);
        g.cx[i] = make_ctx_public(*R[i]);
        grid = std::max(grid, P[i]->grid);
    }
    const size_t smem = group_layout<NA, NB, MT>(g, first_only, false);
    if (!smem) return LGK_EINVAL;
    LGK_CUDA_TRY(launch_k(k_tc_gemm<NA, NB, NT, A_MN, EPI, MT>, dim3(grid), dim3(kThreads), smem, st, pdl, g));
    LGK_LAUNCH_CHECK();
    return LGK_OK;
}

static int maps_for(ResultData& r, TcMaps& M) {
    CaseData& cs = *r.cs;
    int rc;
    if ((rc = make_map(&M.A_k, cs.Ahat.p, cs.n_pad, cs.m_pad, cs.na, 128))) return rc;
    if ((rc = make_map(&M.A_mn, cs.Ahat.p, cs.n_pad, cs.m_pad, cs.na, 64))) return rc;
    if (cs.na == 2) {       // the low BF16 term alone
        const void* lo = static_cast<const char*>(cs.Ahat.p) + (size_t)cs.m_pad * cs.n_pad * 2;
        if ((rc = make_map(&M.Alo_k, lo, cs.n_pad, cs.m_pad, 1, 128))) return rc;
        if ((rc = make_map(&M.Alo_mn, lo, cs.n_pad, cs.m_pad, 1, 64))) return rc;
    } else {
        M.Alo_k = M.A_k;
        M.Alo_mn = M.A_mn;
    }
    if ((rc = make_map(&M.G3, cs.G3.p, cs.m_pad, cs.m_pad, 3, 128))) return rc;
    if ((rc = make_map(&M.R1, r.R1.p, cs.n_pad, r.Kp, 2, r.n_tile))) return rc;
    if ((rc = make_map(&M.rhs, r.rhs.p, cs.m_pad, r.Kp, 3, r.n_tile_s))) return rc;
    if ((rc = make_map(&M.V, r.V.p, cs.m_pad, r.Kp, 2, r.n_tile))) return rc;
    if (r.refine_steps) {
        if ((rc = make_map(&M.S3, cs.S3.p, cs.m_pad, cs.m_pad, 3, 128))) return rc;
        if ((rc = make_map(&M.V3, r.V3.p, cs.m_pad, r.Kp, 3, r.n_tile_s))) return rc;
    }
    return LGK_OK;
}

template <int NA, int NB, int NT, bool A_MN, int EPI, int MT = 1>
static int set_smem_attr() {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<NA, NB, NT, A_MN, EPI, MT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) {
        set_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
        return LGK_ECUDA;
    }
    return LGK_OK;
}

// Outside any stream capture: kernel attributes, TMA descriptors, plans.
int tc_prepare(ResultData& r) {
    CaseData& cs = *r.cs;
    int rc;
    if ((rc = set_smem_attr<1, 2, 2, false, EPI_PARTIAL>())) return rc;
    if ((rc = set_smem_attr<2, 2, 3, false, EPI_PARTIAL>())) return rc;
    if ((rc = set_smem_attr<3, 3, 6, false, EPI_PARTIAL>())) return rc;
    if ((rc = set_smem_attr<1, 2, 2, true, EPI_Q1>())) return rc;
    if ((rc = set_smem_attr<2, 2, 3, true, EPI_Q1>())) return rc;
    if ((rc = set_smem_attr<1, 1, 1, false, EPI_STORE>())) return rc;
    if ((rc = set_smem_attr<1, 1, 1, true, EPI_STORE>())) return rc;
    if ((rc = set_smem_attr<1, 2, 2, false, EPI_PARTIAL, 2>())) return rc;
    if ((rc = set_smem_attr<1, 2, 2, true, EPI_Q1, 2>())) return rc;
    if ((rc = set_smem_attr<1, 1, 1, false, EPI_STORE, 2>())) return rc;
    if ((rc = set_smem_attr<1, 1, 1, true, EPI_STORE, 2>())) return rc;
    if ((rc = maps_for(r, r.maps))) return rc;
    // 256-row tiles for the GEMMs whose A operand is one BF16 term (the
    // one-term form, or A_hi and A_lo with lo_refresh) when two accumulators
    // fit in tensor memory next to each other
    const bool can_wide = (cs.na == 1 || r.refine) && r.n_tile <= 128;
    r.wide = can_wide && (r.force_wide < 0 || r.force_wide == 1);
    // GEMM2's tile height: lgk_params.gemm2_tile_rows (0: as GEMM1), unless
    // the autotuner or a group forces one
    const int p2 = cs.prm.gemm2_tile_rows;
    r.wide2 = r.force_wide2 >= 0 ? can_wide && r.force_wide2 == 1
                                 : (p2 == 128 ? false : p2 == 256 ? can_wide : r.wide);
    const int hm = r.wide ? 2 : 1, hm2 = r.wide2 ? 2 : 1;
    const int mt = cs.m_pad / 128, nt = cs.n_pad / 128;
    if ((rc = build_plan(r.plan1, mt / hm, r.Kp / r.n_tile, cs.n_pad / 64, r.n_tile, false, hm,
                         cs.prm.accum_kblocks)))
        return rc;
    if ((rc = build_plan(r.plan_s, mt, r.Kp / r.n_tile_s, cs.m_pad / 64, r.n_tile_s, false, 1))) return rc;
    if ((rc = build_plan(r.plan2, nt / hm2, r.Kp / r.n_tile, cs.m_pad / 64, r.n_tile, true, hm2))) return rc;
    size_t slots = std::max({(size_t)r.plan1.nseg * r.n_tile * hm, (size_t)r.plan_s.nseg * r.n_tile_s,
                             (size_t)r.plan2.nseg * r.n_tile * hm2});
    return r.part.alloc(slots * 128 * 4);
}

// With lo_refresh the heavy products use A_hi (NA = 1: plane 0 of the
// two-term maps) and the low term comes from tc_gemm1_lo / tc_gemm2_lo.
int tc_gemm1_lo(ResultData& r, bool pdl, bool first_only) {
    if (r.wide)
        return launch<1, 1, 1, false, EPI_STORE, 2>(r.maps.Alo_k, r.maps.R1, r.plan1, r, r.c1.p, pdl,
                                                    first_only);
    return launch<1, 1, 1, false, EPI_STORE>(r.maps.Alo_k, r.maps.R1, r.plan1, r, r.c1.p, pdl, first_only);
}

int tc_gemm2_lo(ResultData& r, bool pdl, bool first_only) {
    if (r.plan2.mt == 2)
        return launch<1, 1, 1, true, EPI_STORE, 2>(r.maps.Alo_mn, r.maps.V, r.plan2, r, r.c2.p, pdl,
                                                   first_only);
    return launch<1, 1, 1, true, EPI_STORE>(r.maps.Alo_mn, r.maps.V, r.plan2, r, r.c2.p, pdl, first_only);
}

int tc_gemm1(ResultData& r, bool pdl) {
    if (r.cs->na == 2 && !r.refine)
        return launch<2, 2, 3, false, EPI_PARTIAL>(r.maps.A_k, r.maps.R1, r.plan1, r, nullptr, pdl);
    if (r.wide) return launch<1, 2, 2, false, EPI_PARTIAL, 2>(r.maps.A_k, r.maps.R1, r.plan1, r, nullptr, pdl);
    return launch<1, 2, 2, false, EPI_PARTIAL>(r.maps.A_k, r.maps.R1, r.plan1, r, nullptr, pdl);
}

int tc_solve(ResultData& r, bool pdl) {
    return launch<3, 3, 6, false, EPI_PARTIAL>(r.maps.G3, r.maps.rhs, r.plan_s, r, nullptr, pdl, false, true);
}

// One EPI_PARTIAL product outside a solve's iteration (the plan check): the
// caller's context (its control block must show work to do) and partial
// buffer.  The kernel needs no predecessor (no programmatic launch).
template <int NA, int NB, int NT, bool A_MN, int EPI, int MT>
static int launch_in(const CUtensorMap& mA, const CUtensorMap& mB, const GemmPlan& P, CaseData& cs,
                     const IterCtx& cx, float* part, cudaStream_t st) {
    TcGroup g;
    memset(&g, 0, sizeof(g));
    g.G = 1;
    g.tmA[0] = mA;
    g.tmB[0] = mB;
    g.a[0] = plan_args(P, part, nullptr, A_MN ? cs.n_pad : cs.m_pad);
    g.cx[0] = cx;
    const size_t smem = group_layout<NA, NB, MT>(g, false, false);
    if (!smem) return LGK_EINVAL;
    LGK_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<NA, NB, NT, A_MN, EPI, MT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
    LGK_CUDA_TRY(launch_k(k_tc_gemm<NA, NB, NT, A_MN, EPI, MT>, dim3(P.grid), dim3(kThreads), smem, st, false, g));
    LGK_LAUNCH_CHECK();
    return LGK_OK;
}

// The plan check's products with exact split operands: A (two BF16 terms,
// K-major for A z1 or MN-major for A^T lam) times three BF16 terms of the
// plans' vectors, 5 products, stream-K segments of at most one k block.
int tc_check_product(CaseData& cs, bool transpose, const CUtensorMap& mA, const CUtensorMap& mB, const GemmPlan& P,
                     const IterCtx& cx, float* part, cudaStream_t st) {
    if (transpose) return launch_in<2, 3, 5, true, EPI_PARTIAL, 1>(mA, mB, P, cs, cx, part, st);
    return launch_in<2, 3, 5, false, EPI_PARTIAL, 1>(mA, mB, P, cs, cx, part, st);
}

// S v for the solve's refinement: the same product shape as the solve.
int tc_sv(ResultData& r, bool pdl) {
    return launch<3, 3, 6, false, EPI_PARTIAL>(r.maps.S3, r.maps.V3, r.plan_s, r, nullptr, pdl);
}

int tc_gemm2(ResultData& r, bool pdl) {
    if (r.cs->na == 2 && !r.refine) return launch<2, 2, 3, true, EPI_Q1>(r.maps.A_mn, r.maps.V, r.plan2, r, r.R1.p, pdl);
    if (r.plan2.mt == 2) return launch<1, 2, 2, true, EPI_Q1, 2>(r.maps.A_mn, r.maps.V, r.plan2, r, r.R1.p, pdl);
    return launch<1, 2, 2, true, EPI_Q1>(r.maps.A_mn, r.maps.V, r.plan2, r, r.R1.p, pdl);
}

}  // namespace lgk

// ------------------------------------------------------------ group launches
// One launch per product over the G solves of a group (run_group checks that
// they share the form: BF16 terms of A, lagged low term, tile height).

namespace lgk {

namespace {
struct GroupOps {
    ResultData* const* R;
    int G;
    const CUtensorMap* a[kMaxGroup];
    const CUtensorMap* b[kMaxGroup];
    const GemmPlan* p[kMaxGroup];
    void* out[kMaxGroup];
};
}  // namespace

#define LGK_GROUP_OPS(EXPR_A, EXPR_B, EXPR_P, EXPR_OUT)      \
    GroupOps o;                                              \
    o.R = R;                                                 \
    o.G = G;                                                 \
    for (int i = 0; i < G && i < kMaxGroup; ++i) {           \
        ResultData& r = *R[i];                               \
        (void)r;                                             \
        o.a[i] = &(EXPR_A);                                  \
        o.b[i] = &(EXPR_B);                                  \
        o.p[i] = &(EXPR_P);                                  \
        o.out[i] = (EXPR_OUT);                               \
    }

int tc_group_gemm1(int G, ResultData* const* R, cudaStream_t st, bool pdl) {
    LGK_GROUP_OPS(r.maps.A_k, r.maps.R1, r.plan1, nullptr);
    const ResultData& r0 = *R[0];
    if (r0.cs->na == 2 && !r0.refine)
        return launch_group<2, 2, 3, false, EPI_PARTIAL, 1>(G, R, o.a, o.b, o.p, o.out, st, pdl, false);
    if (r0.wide) return launch_group<1, 2, 2, false, EPI_PARTIAL, 2>(G, R, o.a, o.b, o.p, o.out, st, pdl, false);
    return launch_group<1, 2, 2, false, EPI_PARTIAL, 1>(G, R, o.a, o.b, o.p, o.out, st, pdl, false);
}

int tc_group_gemm1_lo(int G, ResultData* const* R, cudaStream_t st, bool pdl, bool first_only) {
    LGK_GROUP_OPS(r.maps.Alo_k, r.maps.R1, r.plan1, r.c1.p);
    if (R[0]->wide)
        return launch_group<1, 1, 1, false, EPI_STORE, 2>(G, R, o.a, o.b, o.p, o.out, st, pdl, first_only);
    return launch_group<1, 1, 1, false, EPI_STORE, 1>(G, R, o.a, o.b, o.p, o.out, st, pdl, first_only);
}

int tc_group_solve(int G, ResultData* const* R, cudaStream_t st, bool pdl) {
    LGK_GROUP_OPS(r.maps.G3, r.maps.rhs, r.plan_s, nullptr);
    return launch_group<3, 3, 6, false, EPI_PARTIAL, 1>(G, R, o.a, o.b, o.p, o.out, st, pdl, false);
}

int tc_group_sv(int G, ResultData* const* R, cudaStream_t st, bool pdl) {
    LGK_GROUP_OPS(r.maps.S3, r.maps.V3, r.plan_s, nullptr);
    return launch_group<3, 3, 6, false, EPI_PARTIAL, 1>(G, R, o.a, o.b, o.p, o.out, st, pdl, false);
}

int tc_group_gemm2_lo(int G, ResultData* const* R, cudaStream_t st, bool pdl, bool first_only) {
    LGK_GROUP_OPS(r.maps.Alo_mn, r.maps.V, r.plan2, r.c2.p);
    if (R[0]->plan2.mt == 2)
        return launch_group<1, 1, 1, true, EPI_STORE, 2>(G, R, o.a, o.b, o.p, o.out, st, pdl, first_only);
    return launch_group<1, 1, 1, true, EPI_STORE, 1>(G, R, o.a, o.b, o.p, o.out, st, pdl, first_only);
}

int tc_group_gemm2(int G, ResultData* const* R, cudaStream_t st, bool pdl) {
    LGK_GROUP_OPS(r.maps.A_mn, r.maps.V, r.plan2, r.R1.p);
    const ResultData& r0 = *R[0];
    if (r0.cs->na == 2 && !r0.refine)
        return launch_group<2, 2, 3, true, EPI_Q1, 1>(G, R, o.a, o.b, o.p, o.out, st, pdl, false);
    if (r0.plan2.mt == 2) return launch_group<1, 2, 2, true, EPI_Q1, 2>(G, R, o.a, o.b, o.p, o.out, st, pdl, false);
    return launch_group<1, 2, 2, true, EPI_Q1, 1>(G, R, o.a, o.b, o.p, o.out, st, pdl, false);
}

#undef LGK_GROUP_OPS

}  // namespace lgk
