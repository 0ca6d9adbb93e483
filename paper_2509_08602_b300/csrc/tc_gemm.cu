// Tensor-core GEMMs of one ADMM iteration on sm_103a: tcgen05.mma (BF16 in,
// FP32 accumulate in TMEM), operands staged by TMA (cp.async.bulk.tensor, 128B
// swizzle, no multicast) through an mbarrier ring, warp-specialised CTA:
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM allocator + MMA issuer (one elected lane)
//   warps 2..5  epilogue: tcgen05.ld of the 128 x N accumulator, one row per thread
//
// Output tile: 128 rows of the long dimension (m for GEMM1 and the solve, n
// for GEMM2) x N columns (weightings, N <= 256).  The kernel is persistent and
// stream-K scheduled: the (tile, 64-wide k block) units of a GEMM are cut into
// one contiguous run per CTA, so every SM streams the same number of operand
// blocks; a run is split into segments at tile boundaries, each segment's
// partial sum goes to its own slot (two TMEM accumulators, so the epilogue of
// one segment overlaps the loads and MMAs of the next), and the reduce kernels
// add a tile's slots in k order (deterministic).  Each product A.B of the
// iteration is a sum of BF16 x BF16 terms (exact products, FP32 sums):
//   GEMM1   A . R1         = A_hi.R1_hi + A_hi.R1_lo + A_lo.R1_hi  (3 terms; the
//                            one-term-A form drops A_lo: 2 terms)
//   solve   S^{-1} . rhs   = G_hi.r_hi + G_hi.r_mid + G_mid.r_hi
//                            + G_hi.r_lo + G_mid.r_mid + G_lo.r_hi (6 terms;
//                            S^{-1} and rhs each split into three BF16 parts,
//                            because S amplifies the rounding of its input)
//   GEMM2   A^T . V        = A_hi^T.V_hi + A_hi^T.V_lo + A_lo^T.V_hi (3 or 2 terms)
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

__device__ inline void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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


struct TcArgs {
    const int* cta_seg;   // segments of CTA c: [cta_seg[c], cta_seg[c + 1])
    const int* seg;       // 5 ints per segment: row tile, column tile, kb begin, kb end, slot
    int n_tile;           // columns per tile (multiple of 16, <= 256)
    int tmem_cols;        // columns of one accumulator (power of two >= n_tile); two of them
    int stages;
    int stage_bytes;
    float* part;          // [slot][n_tile][128] segment partial sums
};

constexpr int kThreads = 192;
constexpr int kABytes = 128 * 64 * 2;       // one 128 x 64 BF16 operand tile

template <int NA, int NB, int NT, bool A_MN>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              TcArgs a, Control* ctrl) {
    if (ctrl->n_active == 0 || ctrl->err) return;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int S = a.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * a.stage_bytes);
    // bars: [0, S) stage full, [S, 2S) stage empty, 2S + b accumulator b full,
    // 2S + 2 + b accumulator b drained
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s0 = a.cta_seg[blockIdx.x], s1 = a.cta_seg[blockIdx.x + 1];
    int* err = &ctrl->err;
    const int b_bytes = a.n_tile * 128;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * S + 2; ++s) mbar_init(smem_u32(&bars[s]), 1);
        mbar_init(smem_u32(&bars[2 * S + 2]), 4);     // one arrival per epilogue warp
        mbar_init(smem_u32(&bars[2 * S + 3]), 4);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), 2 * a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer: one continuous stream of k blocks
        bool ok = true;
        int it = 0;
        for (int sg = s0; sg < s1 && ok; ++sg) {
            const int* g = a.seg + 5 * sg;
            const int row0 = g[0] * 128, col0 = g[1] * a.n_tile;
            for (int kb = g[2]; kb < g[3] && ok; ++kb, ++it) {
                const int s = it % S;
                const uint32_t ph = (uint32_t)(it / S) & 1u;
                ok = mbar_wait(smem_u32(&bars[S + s]), ph ^ 1u, err);
                if (!ok) break;
                const uint32_t full = smem_u32(&bars[s]);
                const uint32_t st = smem_u32(smem + (size_t)s * a.stage_bytes);
                mbar_expect_tx(full, (uint32_t)a.stage_bytes);
                const int kx = kb * 64;
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
                const uint32_t sb = st + NA * kABytes;
#pragma unroll
                for (int p = 0; p < NB; ++p) tma_load_3d(sb + p * b_bytes, &tmB, kx, col0, p, full);
            }
        }
        // drain: wait (bounded) for the copies of the last issued stages
        for (int j = max(0, it - S); j < it && ok; ++j)
            ok = mbar_wait(smem_u32(&bars[j % S]), (uint32_t)(j / S) & 1u, err);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = instr_desc(a.n_tile, A_MN);
        bool ok = true;
        int it = 0;
        for (int sg = s0, u = 0; sg < s1; ++sg, ++u) {
            const int* g = a.seg + 5 * sg;
            const int b = u & 1;
            if (ok) ok = mbar_wait(smem_u32(&bars[2 * S + 2 + b]), (uint32_t)((u >> 1) & 1) ^ 1u, err);
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(b * a.tmem_cols);
            for (int kb = g[2]; kb < g[3]; ++kb, ++it) {
                const int s = it % S;
                const uint32_t ph = (uint32_t)(it / S) & 1u;
                if (ok) ok = mbar_wait(smem_u32(&bars[s]), ph, err);
                tc_fence_after();
                const uint32_t st = smem_u32(smem + (size_t)s * a.stage_bytes);
                const uint32_t sb = st + NA * kABytes;
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
                            tc_mma(d, ad, bd, idesc, (kb > g[2] || t > 0 || ks > 0) ? 1u : 0u);
                        }
                    }
                }
                tc_commit(smem_u32(&bars[S + s]));      // frees the stage when its MMAs finish
            }
            tc_commit(smem_u32(&bars[2 * S + b]));      // accumulator b complete
        }
    } else if (warp >= 2) {
        // ---------------- epilogue: accumulator -> segment slot
        const int ew = warp & 3;                        // TMEM lane quarter of this warp
        const int r = ew * 32 + lane;                   // row within the tile
        bool ok = true;
        for (int sg = s0, u = 0; sg < s1; ++sg, ++u) {
            const int b = u & 1;
            if (ok) ok = mbar_wait(smem_u32(&bars[2 * S + b]), (uint32_t)((u >> 1) & 1), err);
            tc_fence_after();
            float* out = a.part + (size_t)a.seg[5 * sg + 4] * a.n_tile * 128 + r;
            const uint32_t base = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(b * a.tmem_cols);
            for (int c0 = 0; c0 < a.n_tile; c0 += 16) {
                float v[16];
                tmem_ld16(base + (uint32_t)c0, v);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) out[(size_t)(c0 + jj) * 128] = ok ? v[jj] : 0.f;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars[2 * S + 2 + b]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * a.tmem_cols);
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
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box,
                    es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
        return LGK_ECUDA;
    }
    return LGK_OK;
}

static constexpr int kSmemLimit = 232448;    // 227 KB opt-in per block

static int smem_extra() { return 1024 + 8 * (2 * 8 + 4) + 16; }

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    }
    return n;
}

// Stream-K plan: the units (column tile, row tile, k block), in that order,
// cut into `grid` contiguous runs of equal length (+-1), each run split into
// segments at tile boundaries.  Depends only on the GEMM's shape.
int build_plan(GemmPlan& P, int rows, int col_tiles, int kb_total, int n_tile) {
    const long long U = (long long)rows * col_tiles * kb_total;
    const int grid = (int)std::min<long long>(sm_count(), U);
    std::vector<int> cta_seg(grid + 1), seg, tile_begin(rows * col_tiles + 1, 0);
    std::vector<std::vector<int>> per_tile(rows * col_tiles);
    int nseg = 0;
    for (int c = 0; c < grid; ++c) {
        cta_seg[c] = nseg;
        long long u0 = U * c / grid, u1 = U * (c + 1) / grid;
        while (u0 < u1) {
            long long tile = u0 / kb_total;
            int kb0 = (int)(u0 % kb_total);
            int kb1 = (int)std::min<long long>(kb_total, kb0 + (u1 - u0));
            int ct = (int)(tile / rows), rt = (int)(tile % rows);
            seg.insert(seg.end(), {rt, ct, kb0, kb1, nseg});
            per_tile[tile].push_back(nseg);
            ++nseg;
            u0 += kb1 - kb0;
        }
    }
    cta_seg[grid] = nseg;
    std::vector<int> tile_slots;
    for (size_t t = 0; t < per_tile.size(); ++t) {
        tile_begin[t] = (int)tile_slots.size();
        tile_slots.insert(tile_slots.end(), per_tile[t].begin(), per_tile[t].end());
    }
    tile_begin[per_tile.size()] = (int)tile_slots.size();
    std::vector<int> all;
    all.insert(all.end(), cta_seg.begin(), cta_seg.end());
    all.insert(all.end(), seg.begin(), seg.end());
    all.insert(all.end(), tile_begin.begin(), tile_begin.end());
    all.insert(all.end(), tile_slots.begin(), tile_slots.end());
    int rc;
    if ((rc = P.buf.alloc(all.size() * 4))) return rc;
    LGK_CUDA_TRY(cudaMemcpy(P.buf.p, all.data(), all.size() * 4, cudaMemcpyHostToDevice));
    const int* d = P.buf.as<int>();
    P.grid = grid;
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

template <int NA, int NB, int NT, bool A_MN>
static int launch(const CUtensorMap& mA, const CUtensorMap& mB, const GemmPlan& P, float* part,
                  Control* ctrl, cudaStream_t st) {
    TcArgs a{};
    a.cta_seg = P.cta_seg;
    a.seg = P.seg;
    a.n_tile = P.n_tile;
    a.part = part;
    a.stage_bytes = NA * kABytes + NB * a.n_tile * 128;
    a.stages = std::min(8, (kSmemLimit - smem_extra()) / a.stage_bytes);
    if (a.stages < 2) {
        set_error("tensor-core GEMM: stage does not fit in shared memory");
        return LGK_EINVAL;
    }
    a.tmem_cols = 32;
    while (a.tmem_cols < a.n_tile) a.tmem_cols <<= 1;
    size_t smem = (size_t)a.stages * a.stage_bytes + smem_extra();
    k_tc_gemm<NA, NB, NT, A_MN><<<P.grid, kThreads, smem, st>>>(mA, mB, a, ctrl);
    LGK_LAUNCH_CHECK();
    return LGK_OK;
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

template <int NA, int NB, int NT, bool A_MN>
static int set_smem_attr() {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<NA, NB, NT, A_MN>,
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
    if ((rc = set_smem_attr<1, 2, 2, false>())) return rc;
    if ((rc = set_smem_attr<2, 2, 3, false>())) return rc;
    if ((rc = set_smem_attr<3, 3, 6, false>())) return rc;
    if ((rc = set_smem_attr<1, 2, 2, true>())) return rc;
    if ((rc = set_smem_attr<2, 2, 3, true>())) return rc;
    if ((rc = maps_for(r, r.maps))) return rc;
    const int mt = cs.m_pad / 128, nt = cs.n_pad / 128;
    if ((rc = build_plan(r.plan1, mt, r.Kp / r.n_tile, cs.n_pad / 64, r.n_tile))) return rc;
    if ((rc = build_plan(r.plan_s, mt, r.Kp / r.n_tile_s, cs.m_pad / 64, r.n_tile_s))) return rc;
    if ((rc = build_plan(r.plan2, nt, r.Kp / r.n_tile, cs.m_pad / 64, r.n_tile))) return rc;
    size_t slots = std::max({(size_t)r.plan1.nseg * r.n_tile, (size_t)r.plan_s.nseg * r.n_tile_s,
                             (size_t)r.plan2.nseg * r.n_tile});
    return r.part.alloc(slots * 128 * 4);
}

int tc_gemm1(ResultData& r) {
    CaseData& cs = *r.cs;
    if (cs.na == 2)
        return launch<2, 2, 3, false>(r.maps.A_k, r.maps.R1, r.plan1, r.part.as<float>(), r.ctrl.as<Control>(), cs.stream);
    return launch<1, 2, 2, false>(r.maps.A_k, r.maps.R1, r.plan1, r.part.as<float>(), r.ctrl.as<Control>(), cs.stream);
}

int tc_solve(ResultData& r) {
    CaseData& cs = *r.cs;
    return launch<3, 3, 6, false>(r.maps.G3, r.maps.rhs, r.plan_s, r.part.as<float>(), r.ctrl.as<Control>(), cs.stream);
}

int tc_gemm2(ResultData& r) {
    CaseData& cs = *r.cs;
    if (cs.na == 2)
        return launch<2, 2, 3, true>(r.maps.A_mn, r.maps.V, r.plan2, r.part.as<float>(), r.ctrl.as<Control>(), cs.stream);
    return launch<1, 2, 2, true>(r.maps.A_mn, r.maps.V, r.plan2, r.part.as<float>(), r.ctrl.as<Control>(), cs.stream);
}

}  // namespace lgk
