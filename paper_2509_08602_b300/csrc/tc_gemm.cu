// Tensor-core GEMMs of one ADMM iteration on sm_103a: tcgen05.mma (BF16 in,
// FP32 accumulate in TMEM), operands staged by TMA (cp.async.bulk.tensor, 128B
// swizzle, no multicast) through an mbarrier ring, warp-specialised CTA:
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM allocator + MMA issuer (one elected lane)
//   warps 2..5  epilogue: tcgen05.ld of the 128 x N accumulator, one row per thread
//
// Output tile: 128 rows of the long dimension (m for GEMM1 and the solve, n
// for GEMM2) x N columns (weightings, N <= 256).  Each product A.B of the
// iteration is a sum of BF16 x BF16 terms (exact products, FP32 sums):
//   GEMM1   A . R1         = A_hi.R1_hi + A_hi.R1_lo + A_lo.R1_hi  (3 terms; the
//                            one-term-A form drops A_lo: 2 terms)
//   solve   S^{-1} . rhs   = G_hi.r_hi + G_hi.r_mid + G_mid.r_hi
//                            + G_hi.r_lo + G_mid.r_mid + G_lo.r_hi (6 terms;
//                            S^{-1} and rhs each split into three BF16 parts,
//                            because S amplifies the rounding of its input)
//   GEMM2   A^T . V        = A_hi^T.V_hi + A_hi^T.V_lo + A_lo^T.V_hi (3 or 2 terms)
// GEMM1 and the solve write split-K partial sums; GEMM2 runs the q1 update
// of the n-block (Eq. admm z- and y-steps in q-form) in its epilogue.
#include <cudaTypedefs.h>

#include <algorithm>
#include <string>

#include "iter_ctx.cuh"
#include "lgk_impl.hpp"

namespace lgk {

// ------------------------------------------------------------ PTX wrappers

__device__ inline uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ inline uint64_t global_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ inline bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~2 s of wall time, records DERR_MBAR_TIMEOUT
// and returns false so the caller can wind down instead of hanging.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_timer();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer() - t0 > 2000000000ull) {
            atomicExch(err, DERR_MBAR_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ inline void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                   uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ inline void tmem_alloc(uint32_t slot_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ inline void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                              uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ inline void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ inline void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor (tcgen05 format): start, leading and stride
// byte offsets in 16-byte units, descriptor version 1, 128-byte swizzle.
__device__ inline uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, M = 128, N = n.
__host__ __device__ constexpr uint32_t instr_desc(int n, bool a_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn_major ? 1u : 0u) << 15) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// term t of an NT-term product: which A part and which B part.
//   NT = 2: A.B_hi + A.B_lo
//   NT = 3: A_hi.B_hi + A_hi.B_lo + A_lo.B_hi
//   NT = 6: all (a, b) with a + b <= 2 over three parts each
// (dropped terms are below 2^-16 resp. 2^-24 of the product, relative).
__host__ __device__ constexpr int term_a(int NT, int t) {
    return NT == 2 ? 0 : NT == 3 ? (t == 2 ? 1 : 0)
                               : (t == 0 || t == 1 || t == 3 ? 0 : (t == 2 || t == 4 ? 1 : 2));
}
__host__ __device__ constexpr int term_b(int NT, int t) {
    return NT == 2 ? t : NT == 3 ? (t == 1 ? 1 : 0)
                               : (t == 0 || t == 2 || t == 5 ? 0 : (t == 1 || t == 4 ? 1 : 2));
}

enum { EPI_PARTIAL = 0, EPI_GEMM2 = 1 };

struct TcArgs {
    int kb_total;       // 64-wide k blocks of the contraction
    int kb_per_split;   // k blocks per CTA along gridDim.z
    int n_tile;         // columns per CTA (multiple of 16, <= 256)
    int tmem_cols;      // power of two >= n_tile
    int stages;
    int stage_bytes;
    float* part;        // EPI_PARTIAL: [split][Kp][rows_pad]
    int rows_pad;
};

constexpr int kThreads = 192;
constexpr int kABytes = 128 * 64 * 2;       // one 128 x 64 BF16 operand tile

template <int NA, int NB, int NT, bool A_MN, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              TcArgs a, IterCtx cx) {
    if (cx.ctrl->n_active == 0 || cx.ctrl->err) return;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int S = a.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * a.stage_bytes);
    // bars[0..S): full, [S..2S): empty, [2S]: accumulator ready
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
    float* ep_smem = reinterpret_cast<float*>(bars + 2 * S + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * 128;
    const int col0 = blockIdx.y * a.n_tile;
    const int split = blockIdx.z;
    const int kb0 = split * a.kb_per_split;
    const int kb1 = min(a.kb_total, kb0 + a.kb_per_split);
    const int nkb = kb1 - kb0;
    int* err = &cx.ctrl->err;
    const int b_bytes = a.n_tile * 128;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * S + 1; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0 && nkb > 0) {
        // ---------------- TMA producer
        bool ok = true;
        for (int it = 0; it < nkb && ok; ++it) {
            int s = it % S;
            uint32_t ph = (uint32_t)(it / S) & 1u;
            ok = mbar_wait(smem_u32(&bars[S + s]), ph ^ 1u, err);
            if (!ok) break;
            uint32_t full = smem_u32(&bars[s]);
            uint32_t st = smem_u32(smem + (size_t)s * a.stage_bytes);
            mbar_expect_tx(full, (uint32_t)a.stage_bytes);
            int kx = (kb0 + it) * 64;
            if (A_MN) {
#pragma unroll
                for (int p = 0; p < NA; ++p) {
                    tma_load_3d(st + p * kABytes, &tmA, row0, kx, p, full);
                    tma_load_3d(st + p * kABytes + kABytes / 2, &tmA, row0 + 64, kx, p, full);
                }
            } else {
#pragma unroll
                for (int p = 0; p < NA; ++p) tma_load_3d(st + p * kABytes, &tmA, kx, row0, p, full);
            }
            uint32_t sb = st + NA * kABytes;
#pragma unroll
            for (int p = 0; p < NB; ++p) tma_load_3d(sb + p * b_bytes, &tmB, kx, col0, p, full);
        }
        // drain: wait (bounded) for the copies of the last issued stages
        int last = nkb;
        for (int it = max(0, last - S); it < last && ok; ++it)
            ok = mbar_wait(smem_u32(&bars[it % S]), (uint32_t)(it / S) & 1u, err);
    } else if (warp == 1 && lane == 0 && nkb > 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = instr_desc(a.n_tile, A_MN);
        bool ok = true;
        for (int it = 0; it < nkb; ++it) {
            int s = it % S;
            uint32_t ph = (uint32_t)(it / S) & 1u;
            if (ok) ok = mbar_wait(smem_u32(&bars[s]), ph, err);
            tc_fence_after();
            uint32_t st = smem_u32(smem + (size_t)s * a.stage_bytes);
            uint32_t sb = st + NA * kABytes;
            if (ok) {
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const uint32_t sa = st + term_a(NT, t) * kABytes;
                    const uint32_t sbt = sb + term_b(NT, t) * b_bytes;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        uint64_t ad = A_MN ? smem_desc(sa + ks * 2048, kABytes / 2, 1024)
                                           : smem_desc(sa + ks * 32, 16, 1024);
                        uint64_t bd = smem_desc(sbt + ks * 32, 16, 1024);
                        tc_mma(tmem, ad, bd, idesc, (it > 0 || t > 0 || ks > 0) ? 1u : 0u);
                    }
                }
            }
            tc_commit(smem_u32(&bars[S + s]));      // frees the stage when the MMAs are done
        }
        tc_commit(smem_u32(&bars[2 * S]));          // accumulator complete
    } else if (warp >= 2) {
        // ---------------- epilogue
        const int ew = warp & 3;                    // TMEM lane quarter of this warp
        const int row = row0 + ew * 32 + lane;
        const int et = threadIdx.x - 64;            // 0..127
        bool ok = nkb > 0 && mbar_wait(smem_u32(&bars[2 * S]), 0u, err);
        tc_fence_after();
        if (EPI == EPI_PARTIAL) {
            float* out = a.part + ((size_t)split * cx.Kp + col0) * a.rows_pad + row;
            for (int c0 = 0; c0 < a.n_tile; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj)
                    out[(size_t)(c0 + jj) * a.rows_pad] = ok ? v[jj] : 0.f;
            }
        } else {
            // GEMM2 epilogue: q1 update of the n-block for this row p = row
            const bool check = is_check_iter(cx.ctrl, cx.check_every, cx.tol);
            float* acc = ep_smem;                   // [n_tile][5] residual sums
            for (int e = et; e < a.n_tile * 5; e += 128) acc[e] = 0.f;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            const int p = row;
            const int sl = cx.col_slot[p];
            const float c = cx.c_slot[sl];
            __nv_bfloat16* R1 = reinterpret_cast<__nv_bfloat16*>(a.part);   // R1 hi/lo buffer
            for (int c0 = 0; c0 < a.n_tile; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int j = col0 + c0 + jj;
                    const size_t o = (size_t)j * cx.n_pad + p;
                    const float u = cx.utab[j * cx.n_slot + sl];
                    const float cr = c * cx.inv_rho[j];
                    Q1Update q = q1_update(cx.q1[o], ok ? v[jj] : 0.f, u, cr);
                    if (cx.active[j]) cx.q1[o] = q.qn;
                    __nv_bfloat16 hi, lo;
                    split_bf16(q.r1, hi, lo);
                    R1[o] = hi;
                    R1[(size_t)cx.Kp * cx.n_pad + o] = lo;
                    if (check) {
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            float s = q.res[k];
#pragma unroll
                            for (int of = 16; of > 0; of >>= 1) s += __shfl_xor_sync(0xffffffffu, s, of);
                            if (lane == 0) atomicAdd(&acc[(c0 + jj) * 5 + k], s);
                        }
                    }
                }
            }
            if (check) {
                asm volatile("bar.sync 1, 128;" ::: "memory");
                for (int e = et; e < a.n_tile * 5; e += 128) {
                    int jj = e / 5, k = e % 5;
                    cx.resid[((size_t)blockIdx.x * cx.Kp + col0 + jj) * 5 + k] = (double)acc[e];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, a.tmem_cols);
    }
}

// ------------------------------------------------------------- host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
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
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims,
                    strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
        return LGK_ECUDA;
    }
    return LGK_OK;
}

static constexpr int kSmemLimit = 232448;    // 227 KB opt-in per block

static int smem_extra(int n_tile) { return 1024 + 8 * 20 + 16 + n_tile * 5 * 4; }

template <int NA, int NB, int NT, bool A_MN, int EPI>
static int launch(const CUtensorMap& mA, const CUtensorMap& mB, TcArgs a, const IterCtx& cx,
                  dim3 grid, cudaStream_t st) {
    a.stage_bytes = NA * kABytes + NB * a.n_tile * 128;
    int extra = smem_extra(a.n_tile);
    a.stages = std::min(8, (kSmemLimit - extra) / a.stage_bytes);
    if (a.stages < 2) {
        set_error("tensor-core GEMM: stage does not fit in shared memory");
        return LGK_EINVAL;
    }
    a.tmem_cols = 32;
    while (a.tmem_cols < a.n_tile) a.tmem_cols <<= 1;
    size_t smem = (size_t)a.stages * a.stage_bytes + extra;
    auto kern = k_tc_gemm<NA, NB, NT, A_MN, EPI>;
    kern<<<grid, kThreads, smem, st>>>(mA, mB, a, cx);
    LGK_LAUNCH_CHECK();
    return LGK_OK;
}

// split-K factor: enough CTAs to cover the SMs about once, every split at
// least 4 k blocks; independent of K so a column's sums never depend on the
// batch it is solved in.
int plan_splits(int kblocks, int row_tiles, int n_tiles) {
    (void)n_tiles;
    int s = std::max(1, 148 / std::max(1, row_tiles));
    s = std::min(s, std::max(1, kblocks / 4));
    // make every split non-empty
    int per = (kblocks + s - 1) / s;
    s = (kblocks + per - 1) / per;
    return s;
}

static int maps_for(ResultData& r, TcMaps& M) {
    CaseData& cs = *r.cs;
    int rc;
    if ((rc = make_map(&M.A_k, cs.Ahat.p, cs.n_pad, cs.m_pad, cs.na, 128))) return rc;
    if ((rc = make_map(&M.A_mn, cs.Ahat.p, cs.n_pad, cs.m_pad, cs.na, 64))) return rc;
    if ((rc = make_map(&M.G3, cs.G3.p, cs.m_pad, cs.m_pad, 3, 128))) return rc;
    if ((rc = make_map(&M.R1, r.R1.p, cs.n_pad, r.Kp, 2, r.n_tile))) return rc;
    if ((rc = make_map(&M.rhs, r.rhs.p, cs.m_pad, r.Kp, 3, r.n_tile_s))) return rc;
    if ((rc = make_map(&M.V, r.V.p, cs.m_pad, r.Kp, 2, r.n_tile))) return rc;
    return LGK_OK;
}

static int ensure_maps(ResultData& r) {
    if (r.maps_ready) return LGK_OK;
    int rc = maps_for(r, r.maps);
    r.maps_ready = rc == LGK_OK;
    return rc;
}

template <int NA, int NB, int NT, bool A_MN, int EPI>
static int set_smem_attr() {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<NA, NB, NT, A_MN, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) {
        set_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
        return LGK_ECUDA;
    }
    return LGK_OK;
}

// Outside any stream capture: kernel attributes and the TMA descriptors.
int tc_prepare(ResultData& r) {
    int rc;
    if ((rc = set_smem_attr<1, 2, 2, false, EPI_PARTIAL>())) return rc;
    if ((rc = set_smem_attr<2, 2, 3, false, EPI_PARTIAL>())) return rc;
    if ((rc = set_smem_attr<3, 3, 6, false, EPI_PARTIAL>())) return rc;
    if ((rc = set_smem_attr<1, 2, 2, true, EPI_GEMM2>())) return rc;
    if ((rc = set_smem_attr<2, 2, 3, true, EPI_GEMM2>())) return rc;
    return ensure_maps(r);
}

int tc_gemm1(ResultData& r) {
    int rc;
    if ((rc = ensure_maps(r))) return rc;
    CaseData& cs = *r.cs;
    TcArgs a{};
    a.kb_total = cs.n_pad / 64;
    a.kb_per_split = (a.kb_total + r.splits1 - 1) / r.splits1;
    a.n_tile = r.n_tile;
    a.part = r.part.as<float>();
    a.rows_pad = cs.m_pad;
    dim3 grid(cs.m_pad / 128, r.Kp / r.n_tile, r.splits1);
    if (cs.na == 2)
        return launch<2, 2, 3, false, EPI_PARTIAL>(r.maps.A_k, r.maps.R1, a, make_ctx_public(r), grid, cs.stream);
    return launch<1, 2, 2, false, EPI_PARTIAL>(r.maps.A_k, r.maps.R1, a, make_ctx_public(r), grid, cs.stream);
}

int tc_solve(ResultData& r) {
    int rc;
    if ((rc = ensure_maps(r))) return rc;
    CaseData& cs = *r.cs;
    TcArgs a{};
    a.kb_total = cs.m_pad / 64;
    a.kb_per_split = (a.kb_total + r.splits_s - 1) / r.splits_s;
    a.n_tile = r.n_tile_s;
    a.part = r.part.as<float>();
    a.rows_pad = cs.m_pad;
    dim3 grid(cs.m_pad / 128, r.Kp / r.n_tile_s, r.splits_s);
    return launch<3, 3, 6, false, EPI_PARTIAL>(r.maps.G3, r.maps.rhs, a, make_ctx_public(r), grid, cs.stream);
}

int tc_gemm2(ResultData& r) {
    int rc;
    if ((rc = ensure_maps(r))) return rc;
    CaseData& cs = *r.cs;
    TcArgs a{};
    a.kb_total = cs.m_pad / 64;
    a.kb_per_split = a.kb_total;
    a.n_tile = r.n_tile;
    a.part = reinterpret_cast<float*>(r.R1.p);      // epilogue output: R1 hi/lo
    a.rows_pad = cs.n_pad;
    dim3 grid(cs.n_pad / 128, r.Kp / r.n_tile, 1);
    if (cs.na == 2)
        return launch<2, 2, 3, true, EPI_GEMM2>(r.maps.A_mn, r.maps.V, a, make_ctx_public(r), grid, cs.stream);
    return launch<1, 2, 2, true, EPI_GEMM2>(r.maps.A_mn, r.maps.V, a, make_ctx_public(r), grid, cs.stream);
}

}  // namespace lgk
