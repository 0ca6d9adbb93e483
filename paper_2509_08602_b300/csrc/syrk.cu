// S = I + A A^T on the tensor cores (the Schur complement of the x-step,
// Sec. 2.B, formed once per case; the paper counts its factorisation as the
// constant overhead of a case).
//
// A is the matrix the iterations use, held as BF16 terms (A = hi, or hi + lo
// exactly).  Every BF16 x BF16 product is exact in FP32, so the only
// rounding is in the sums: each output tile accumulates the products of
// kKC k-blocks (64 columns of A each) in tensor memory in FP32, and the
// epilogue adds these short chunk sums into FP64 registers.  The entries of S
// come out with about 1e-6 relative error (FP32 sums of at most
// kKC * 4 * 3 partial products) instead of the 1e-16 of an FP64 product; the
// iterations' explicit S^{-1} (three BF16 terms, FP32 sums) is further off
// than that, and with solve_refine the split's constraint error is
// dS v ~ 1e-6 |S| |v|, far below the residual tolerance.
//
// Tiles: 128 rows x 64 columns of the lower triangle (every tile that meets
// it, so every 64 x 64 diagonal block is written whole, as the blocked
// Cholesky expects); persistent CTAs take tiles round-robin.  Warp roles:
// 0 TMA producer, 1 TMEM allocator + MMA issuer, 2..5 epilogue (one per TMEM
// lane quarter, one row per thread, 64 FP64 accumulators).
#include <algorithm>
#include <string>
#include <vector>

#include "lgk_impl.hpp"
#include "tc_ptx.cuh"

namespace lgk {

constexpr int kSyrkN = 64;            // columns of S per tile
constexpr int kSyrkStages = 4;
constexpr int kSyrkKC = 2;            // k blocks summed in tensor memory per FP64 add
constexpr int kSyrkThreads = 192;
constexpr int kSyrkABytes = 128 * 64 * 2;   // one 128-row BF16 tile of a k block
constexpr int kSyrkBBytes = kSyrkN * 64 * 2;

__device__ inline void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ inline void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// tiles[t] = (row tile, column tile); S row-major FP64 [m_pad][ld]
template <int NA>
__global__ void __launch_bounds__(kSyrkThreads, 1)
    k_tc_syrk(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const int2* __restrict__ tiles, int n_tiles, int kb_total, double* __restrict__ S, int ld,
              int* err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int stage_bytes = NA * (kSyrkABytes + kSyrkBBytes);
    constexpr int S_ = kSyrkStages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S_ * stage_bytes);
    // bars: [0, S) full, [S, 2S) empty, 2S + b accumulator b full, 2S + 2 + b drained
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S_ + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_chunks = (kb_total + kSyrkKC - 1) / kSyrkKC;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * S_ + 2; ++s) mbar_init(smem_u32(&bars[s]), 1);
        for (int b = 0; b < 2; ++b) mbar_init(smem_u32(&bars[2 * S_ + 2 + b]), 4);   // epilogue warps
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), 2 * kSyrkN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        bool ok = true;
        int it = 0;
        for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const int2 tl = tiles[t];
            for (int kb = 0; kb < kb_total && ok; ++kb, ++it) {
                const int s = it % S_;
                const uint32_t ph = (uint32_t)(it / S_) & 1u;
                ok = mbar_wait(smem_u32(&bars[S_ + s]), ph ^ 1u, err);
                if (!ok) break;
                const uint32_t full = smem_u32(&bars[s]);
                const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
                mbar_expect_tx(full, (uint32_t)stage_bytes);
#pragma unroll
                for (int p = 0; p < NA; ++p) {
                    tma_load_3d(st + p * kSyrkABytes, &tmA, kb * 64, tl.x * 128, p, full);
                    tma_load_3d(st + NA * kSyrkABytes + p * kSyrkBBytes, &tmB, kb * 64, tl.y * kSyrkN, p, full);
                }
            }
        }
        for (int j = max(0, it - S_); j < it && ok; ++j)
            ok = mbar_wait(smem_u32(&bars[j % S_]), (uint32_t)(j / S_) & 1u, err);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer: per chunk of kKC k blocks, a fresh accumulator
        const uint32_t idesc = instr_desc(kSyrkN, false);
        bool ok = true;
        int it = 0, u = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            for (int c = 0; c < n_chunks; ++c, ++u) {
                const int b = u & 1;
                if (ok) ok = mbar_wait(smem_u32(&bars[2 * S_ + 2 + b]), (uint32_t)((u >> 1) & 1) ^ 1u, err);
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * kSyrkN);
                const int kb1 = min(kb_total, (c + 1) * kSyrkKC);
                for (int kb = c * kSyrkKC; kb < kb1; ++kb, ++it) {
                    const int s = it % S_;
                    const uint32_t ph = (uint32_t)(it / S_) & 1u;
                    if (ok) ok = mbar_wait(smem_u32(&bars[s]), ph, err);
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
                    if (ok) {
                        // products hi.hi (+ hi.lo + lo.hi): the lo.lo term is below 2^-16 of the others
#pragma unroll
                        for (int q = 0; q < (NA == 2 ? 3 : 1); ++q) {
                            const int pa = q == 2 ? 1 : 0, pb = q == 1 ? 1 : 0;
                            const uint32_t sa = st + pa * kSyrkABytes;
                            const uint32_t sb = st + NA * kSyrkABytes + pb * kSyrkBBytes;
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks)
                                tc_mma(d, smem_desc(sa + ks * 32, 16, 1024), smem_desc(sb + ks * 32, 16, 1024),
                                       idesc, (kb > c * kSyrkKC || q > 0 || ks > 0) ? 1u : 0u);
                        }
                    }
                    tc_commit(smem_u32(&bars[S_ + s]));
                }
                tc_commit(smem_u32(&bars[2 * S_ + b]));
            }
        }
    } else if (warp >= 2) {
        // ---------------- epilogue: FP64 sums of the chunks, one row per thread
        const int ew = warp & 3;
        const int r = ew * 32 + lane;
        bool ok = true;
        int u = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            const int2 tl = tiles[t];
            double acc[kSyrkN];
#pragma unroll
            for (int c = 0; c < kSyrkN; ++c) acc[c] = 0.0;
            for (int c = 0; c < n_chunks; ++c, ++u) {
                const int b = u & 1;
                if (ok) ok = mbar_wait(smem_u32(&bars[2 * S_ + b]), (uint32_t)((u >> 1) & 1), err);
                tc_fence_after();
                const uint32_t base = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(b * kSyrkN);
#pragma unroll
                for (int c0 = 0; c0 < kSyrkN; c0 += 16) {
                    float v[16];
                    tmem_ld16(base + (uint32_t)c0, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 16; ++k) acc[c0 + k] += ok ? (double)v[k] : 0.0;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bars[2 * S_ + 2 + b]));
            }
            const int i = tl.x * 128 + r;
            double* row = S + (size_t)i * ld + tl.y * kSyrkN;
#pragma unroll
            for (int c = 0; c < kSyrkN; ++c) row[c] = acc[c] + (i == tl.y * kSyrkN + c ? 1.0 : 0.0);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * kSyrkN);
    }
}

// Host: S (FP64, m_pad x m_pad, row-major, lower 64-blocks and every diagonal
// 64 x 64 block written) = I + A A^T from the case's BF16 terms of A.
int tc_syrk(CaseData& cs, double* S, int* err) {
    const int na = cs.na;
    if (na < 1 || na > 2) {
        set_error("tc_syrk: the case has no BF16 terms of A");
        return LGK_EINVAL;
    }
    const int m_pad = cs.m_pad, n_pad = cs.n_pad;
    CUtensorMap mA, mB;
    int rc;
    if ((rc = make_tma_map(&mA, cs.Ahat.p, n_pad, m_pad, na, 128))) return rc;
    if ((rc = make_tma_map(&mB, cs.Ahat.p, n_pad, m_pad, na, kSyrkN))) return rc;
    std::vector<int2> tiles;
    for (int rt = 0; rt < m_pad / 128; ++rt)
        for (int ct = 0; ct * kSyrkN <= rt * 128 + 127; ++ct) tiles.push_back(make_int2(rt, ct));
    DevBuf td;
    if ((rc = td.alloc(tiles.size() * sizeof(int2)))) return rc;
    LGK_CUDA_TRY(cudaMemcpyAsync(td.p, tiles.data(), td.bytes, cudaMemcpyHostToDevice, cs.stream));
    const int stage_bytes = na * (kSyrkABytes + kSyrkBBytes);
    const size_t smem = 1024 + (size_t)kSyrkStages * stage_bytes + 8 * (2 * kSyrkStages + 4) + 16;
    const int grid = std::min<int>(sm_count(), (int)tiles.size());
    const int kb = n_pad / 64;
    if (na == 2) {
        LGK_CUDA_TRY(cudaFuncSetAttribute(k_tc_syrk<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_tc_syrk<2><<<grid, kSyrkThreads, smem, cs.stream>>>(mA, mB, td.as<int2>(), (int)tiles.size(), kb, S,
                                                              m_pad, err);
    } else {
        LGK_CUDA_TRY(cudaFuncSetAttribute(k_tc_syrk<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_tc_syrk<1><<<grid, kSyrkThreads, smem, cs.stream>>>(mA, mB, td.as<int2>(), (int)tiles.size(), kb, S,
                                                              m_pad, err);
    }
    LGK_LAUNCH_CHECK();
    LGK_CUDA_TRY(cudaStreamSynchronize(cs.stream));      // td is freed on return
    return LGK_OK;
}

}  // namespace lgk
