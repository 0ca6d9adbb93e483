// Internal definitions shared by the liblgk translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/lgk.h"

namespace lgk {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
void count_launch(long long n = 1);

struct Status {
    int code = LGK_OK;
};

#define LGK_CUDA_TRY(expr)                                                      \
    do {                                                                        \
        cudaError_t _e = (expr);                                                \
        if (_e != cudaSuccess) {                                                \
            ::lgk::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e) \
                             + " (" + __FILE__ + ":" + std::to_string(__LINE__) \
                             + ")");                                            \
            return _e == cudaErrorMemoryAllocation ? LGK_ENOMEM : LGK_ECUDA;    \
        }                                                                       \
    } while (0)

#define LGK_LAUNCH_CHECK()                                                      \
    do {                                                                        \
        ::lgk::count_launch();                                                  \
        cudaError_t _e = cudaGetLastError();                                    \
        if (_e != cudaSuccess) {                                                \
            ::lgk::set_error(std::string("kernel launch: ") +                   \
                             cudaGetErrorString(_e) + " (" + __FILE__ + ":" +   \
                             std::to_string(__LINE__) + ")");                   \
            return LGK_ECUDA;                                                   \
        }                                                                       \
    } while (0)

// ------------------------------------------------------------ small helpers
__host__ __device__ inline long long round_up(long long x, long long r) {
    return (x + r - 1) / r * r;
}

// Programmatic dependent launch (kernels of one iteration launched with
// cudaLaunchAttributeProgrammaticStreamSerialization).  pdl_trigger lets the
// next kernel of the stream start launching (its CTAs run their set-up on SMs
// this kernel has left); pdl_wait blocks until the previous kernel of the
// stream has completed and its writes are visible.  Without a programmatic
// predecessor the wait returns at once.
__device__ inline void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ inline void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `kern` on `st`, allowed to overlap the previous kernel's tail when
// `pdl` (the kernel must call pdl_wait before reading that kernel's output).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// The same with an L2 access-policy window (lines of [base, base + bytes)
// marked persisting, when a persisting carve-out is set); win may be null.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k_win(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                bool pdl, const cudaAccessPolicyWindow* win, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (pdl) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    if (win) {
        attr[na].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[na].val.accessPolicyWindow = *win;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Device-side error codes written into Control::err.
enum DeviceError : int {
    DERR_NONE = 0,
    DERR_MBAR_TIMEOUT = 1,   // a bounded mbarrier wait in a tensor-core GEMM ran out
    DERR_NOT_PD = 2,         // non-positive pivot in the FP64 Cholesky
    DERR_BAD_SHAPE = 3,      // a kernel was launched with a shape it cannot handle
};

// Control block of one solve (device memory).
struct Control {
    int iter;        // iterations completed
    int n_active;    // columns still iterating
    int max_iter;
    int err;         // DeviceError
    int ticket;      // blocks of the finalize kernel done this iteration
};

// Point-class slots of the A columns: per target k: TS=3k, TI=3k+1, R=3k+2;
// then LD1, LD2, OAR, BOT (coupling columns), PAD (zero padding).
__host__ __device__ inline int slot_ld1(int n_targets) { return 3 * n_targets; }
__host__ __device__ inline int slot_ld2(int n_targets) { return 3 * n_targets + 1; }
__host__ __device__ inline int slot_oar(int n_targets) { return 3 * n_targets + 2; }
__host__ __device__ inline int slot_bot(int n_targets) { return 3 * n_targets + 3; }
__host__ __device__ inline int slot_pad(int n_targets) { return 3 * n_targets + 4; }
__host__ __device__ inline int n_slots(int n_targets) { return 3 * n_targets + 5; }
constexpr int kMaxTargets = 64;      // keeps slot ids below 255

// Exact round-to-nearest-even of an FP64 value to bfloat16 (8 significant
// bits, FP32 exponent range, subnormal spacing 2^-133).  Normal range
// (|x| >= 2^-126): round the 52-bit fraction to its top 7 bits on the bit
// pattern (add half an ulp minus one, plus the kept lsb, then clear the 45
// dropped bits; a carry moves into the exponent correctly).  Below 2^-126:
// scale to an integer significand, round with rint (ties to even), scale
// back.  Either result has at most 8 significant bits and lies in float
// range (or overflows to inf), so the float and bf16 conversions are exact.
__device__ inline __nv_bfloat16 bf16_from_double(double x) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int bexp = (int)((bits >> 52) & 0x7ff);
    if (bexp != 0x7ff && bexp >= 1023 - 126) {
        bits += 0x00000FFFFFFFFFFFull + ((bits >> 45) & 1ull);
        bits &= ~0x00001FFFFFFFFFFFull;
        const double r = __longlong_as_double((long long)bits);
        const float rf = fabs(r) >= 0x1p128 ? (r < 0 ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000))
                                            : (float)r;
        return __float2bfloat16_rn(rf);
    }
    if (x == 0.0 || !isfinite(x)) return __float2bfloat16_rn((float)x);
    double ax = fabs(x);
    int e;
    frexp(ax, &e);           // ax = f 2^e, f in [0.5, 1)
    e -= 1;                  // ax in [2^e, 2^(e+1))
    if (e < -126) e = -126;
    double q = ldexp(1.0, e - 7);
    double r = rint(ax / q) * q;
    float rf = r >= 0x1p128 ? __int_as_float(0x7f800000) : (float)r;
    return __float2bfloat16_rn(x < 0 ? -rf : rf);
}

}  // namespace lgk
