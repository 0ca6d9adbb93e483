// Host-side objects behind the opaque lgk_case / lgk_result handles.
#pragma once

#include <cublas_v2.h>

#include <atomic>
#include <condition_variable>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lgk_common.cuh"

namespace lgk {

// Device buffer owned by a case or result.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { if (p) cudaFree(p); }
    int alloc(size_t n);
    template <class T> T* as() const { return static_cast<T*>(p); }
};

struct CheckTC;   // tensor-core plan check of a case (check.cu)

// S's three BF16 terms are kept when a solve may refine its x-update: from
// its start (solve_refine) or after refine_after iterations.
inline bool keeps_s3(const lgk_params& p) { return p.solve_refine > 0 || p.refine_after > 0; }

struct CaseData {
    lgk_params prm{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cublasHandle_t cublas = nullptr;
    DevBuf cublas_ws;

    // problem sizes (Appendix A): m = 24N + N rows, n = P + 8N columns
    int n_iso = 0, n_pts = 0, n_beams = 0, m = 0, n = 0;
    int m_pad = 0, n_pad = 0;              // multiples of 256
    int n_targets = 0, n_oars = 0, n_slot = 0;
    double beta = 1.0;
    double a_norm = 0.0;                   // ||A||_2 of the iterations' A (power iteration on S)
    std::vector<int> slot_count;           // points per slot (TS/TI/R per target, LD1, LD2, OAR)
    std::vector<uint8_t> slot_host;        // slot of every point [n_pts]
    std::vector<double> q_area, q_vol, d_presc;
    std::vector<float> c_of_slot;          // c per slot (Appendix A: -1, -1, +1, +1, +1, 0)

    DevBuf col_slot;   // uint8 [n_pad]
    DevBuf Dr;         // double [m_pad] row scale D_r (1 on padding rows)
    DevBuf A32;        // float [m_pad][n_pad]           (LGK_PREC_FP32)
    DevBuf Ahat;       // bf16 [na][m_pad][n_pad]: A = hi (+ lo)   (BF16 forms)
    int na = 0;        // BF16 terms of A: 1 (LGK_PREC_BF16), 2 (LGK_PREC_BF16X3)
    DevBuf G32;        // float [m_pad][m_pad] S^{-1}    (LGK_PREC_FP32)
    DevBuf G3;         // bf16 [3][m_pad][m_pad] S^{-1} = hi + mid + lo (BF16 forms)
    DevBuf S3;         // bf16 [3][m_pad][m_pad] S = hi + mid + lo (BF16 forms, keeps_s3)
    DevBuf ctrl_setup; // int [4] device error flags during set-up
    std::atomic<int> async_busy{0};   // an asynchronous solve of this case is running
    std::unique_ptr<CheckTC> chk_tc;  // plans, maps and buffers of the plan check, made on first use
    // GEMM configurations chosen by the autotuner (lgk_params.autotune), per
    // column count Kp: (256-row tiles for GEMM1 in bit 0 and for GEMM2 in
    // bit 1, solve column tile)
    std::map<int, std::pair<int, int>> tuned;
    std::mutex tune_mu;
    size_t bytes_held() const;
    ~CaseData();
};

// TMA descriptors of one solve's operands (128B-swizzled BF16 tiles).
struct TcMaps {
    CUtensorMap A_k;    // A terms, K-major tiles 128 rows x 64 columns (GEMM1)
    CUtensorMap A_mn;   // A terms, tiles 64 rows x 64 columns read MN-major (GEMM2)
    CUtensorMap G3;     // S^{-1} hi/mid/lo, 128 x 64 tiles (solve)
    CUtensorMap R1, rhs, V;   // hi/lo iterates, n_tile x 64 tiles
    CUtensorMap Alo_k, Alo_mn;   // A's low BF16 term alone (lo_refresh products)
    CUtensorMap S3, V3;          // S hi/mid/lo (128 x 64 tiles) and v's three terms (refinement)
};

// Stream-K work plan of one tensor-core GEMM (device int arrays, see
// build_plan): per CTA its segments, per segment (row tile, column tile,
// k begin, k end, slot), per output tile the slots that cover it in k order.
struct GemmPlan {
    DevBuf buf;
    int grid = 0, nseg = 0, rows = 0, col_tiles = 0, n_tile = 0;
    int mt = 1;                     // 128-row sub-tiles per output tile (tile height 128 mt)
    const int* cta_seg = nullptr;
    const int* seg = nullptr;
    const int* tile_begin = nullptr;
    const int* tile_slots = nullptr;
    int* tile_count = nullptr;      // per tile: segments done in the running launch
};

// The plan check on the tensor cores (check.cu): its two products' plans
// (stream-K segments of one k block), TMA maps, split operands of up
// to kCheckCols plans, partial sums and a control block showing work to do.
constexpr int kCheckCols = 16;
struct CheckTC {
    GemmPlan az, atl;
    DevBuf part, ctrl, z3, l3;
    CUtensorMap mA_k, mA_mn, mZ, mL;
};

struct ResultData {
    std::shared_ptr<CaseData> cs;
    TcMaps maps;
    GemmPlan plan1, plan_s, plan2;    // GEMM1, solve, GEMM2
    int K = 0, Kp = 0, n_tile = 0, n_tile_s = 0;   // column tiles: GEMMs, solve
    double tol = 0.0;
    int max_iter = 0;

    DevBuf q1, q2;            // float [Kp][n_pad], [Kp][m_pad]
    DevBuf R1;                // FP32: float [Kp][n_pad]; BF16: bf16 [2][Kp][n_pad]
    DevBuf rhs, V;            // FP32: float [Kp][m_pad]; BF16: rhs bf16 [3][Kp][m_pad], V [2][Kp][m_pad]
    DevBuf W;                 // FP32 only: float [Kp][n_pad] (A^T V before its epilogue)
    DevBuf part;              // float segment partial sums [slot][n_tile][128] (BF16 forms), or
                              // one GEMM output [Kp][rows] (FP32 form)
    DevBuf utab;              // float [Kp][n_slot] upper bounds u per slot
    bool refine = false;      // lo_refresh: heavy products with A_hi, lo products lagged
    bool wide = false;        // GEMM1 / GEMM2 (and the lo products) on 256-row tiles
    int force_wide = -1;      // autotuner: -1 the default rule, 0 / 1 forced (where allowed)
    bool wide2 = false;       // GEMM2 (and its low-term product) on 256-row tiles
    int force_wide2 = -1;     // autotuner / group: -1 lgk_params.gemm2_tile_rows, 0 / 1 forced
    DevBuf c1, c2;            // float [Kp][m_pad] lo R1_hi, [Kp][n_pad] lo^T V_hi (last full iteration)
    int refine_steps = 0;     // solve refinement steps per iteration (lgk_params.solve_refine)
    bool l2_keep = false;     // l2_keep_inverse: the solve's S^{-1} loads persist in an L2 carve-out
    cudaAccessPolicyWindow l2win{};   // the window over S^{-1}'s terms
    DevBuf rhs32, rv, V3;     // refinement: rhs FP32 [Kp][m_pad], v so far FP32, v as bf16 [3][Kp][m_pad]
    DevBuf mask;              // uint32 [n_pad][mask_words] point selection, when given
    int mask_words = 0;       // 0: every point in every column
    DevBuf colp;              // float [4][Kp]: rho, 1/rho, w_BOT, unused
    DevBuf active, iters;     // int [Kp]
    DevBuf ctrl;              // Control
    DevBuf resid;             // double [n_resid_blocks][Kp][5] residual partial sums
    DevBuf stats;             // double [3][Kp]: rel_pri, rel_dual, obj
    std::vector<double> u64;  // host [Kp][n_slot]: each column's bounds u in FP64 (the FP64 check)
    std::vector<double> wb64; // host [Kp]: each column's w_BOT in FP64
    std::vector<float> colp_h;// host copy of colp (rho, 1/rho, w_BOT as the iteration holds them)
    DevBuf chk;               // device temporaries of the FP64 check (run_check)

    // asynchronous solve (lgk_solve_weightings_async): the worker thread that
    // runs it, its outcome, and a cancel request checked between graph replays
    std::thread worker;
    std::mutex amu;
    std::condition_variable acv;
    bool running = false;
    bool waited = true;       // false from the async start until lgk_wait succeeds
    int async_rc = LGK_OK;
    std::string async_err;
    std::atomic<bool> cancel{false};
    int n_resid_n = 0, n_resid_m = 0;     // residual partial blocks from the n- and m-blocks

    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    std::vector<int> prof_class;             // kernel classes of one iteration, launch order
    std::vector<cudaEvent_t> prof_ev;        // prof_class.size() + 1 per captured iteration
    std::vector<char> prof_ran;              // per captured iteration and class slot: launched
    double prof_ms[LGK_K_COUNT] = {0};
    long long prof_n[LGK_K_COUNT] = {0};
    ~ResultData();
};

// set-up (setup.cu)
int setup_case(CaseData& cs, const lgk_case_desc& d);

// Result of one weighting of a stream (host memory, valid during the call).
struct StreamOut {
    const double* t;         // n_beams sector times (unscaled)
    const double* tau;       // n_iso isocenter times
    int iters;
    double obj, rel_pri, rel_dual;
    bool converged;
    const double* check;     // LGK_CHECK_COUNT values of the FP64 check, or null
};

// Streaming solve (lgk_solve_stream): K_total weightings admitted into the
// columns of one solve as earlier ones stop; results are written per
// weighting (host arrays, each may be null).  With `pull` set (serving), the
// weightings come from it instead of W / rho and the results go to `done`.
struct StreamSpec {
    int K_total = 0;
    const double* W = nullptr;       // K_total x 4
    const double* rho = nullptr;     // K_total
    int max_iter = 0;                // per weighting
    double *t = nullptr, *tau = nullptr, *obj = nullptr, *rel_pri = nullptr, *rel_dual = nullptr;
    int* iters = nullptr;
    uint8_t* converged = nullptr;
    double* check = nullptr;         // K_total x LGK_CHECK_COUNT (FP64 check per weighting)
    // dynamic source: pull(w[4], &rho, &tag, block) returns 1 (a weighting),
    // 0 (none now; only when !block) or -1 (closed and drained)
    std::function<int(double*, double*, long long*, bool)> pull;
    std::function<void(long long, const StreamOut&)> done;
    bool want_check = false;         // run the FP64 check for `done`
    int n_initial = -1;              // columns filled at the start (run_solve's W rows); -1: all
    const long long* initial_tags = nullptr;
};

// one solve (iter.cu); with `stream`, W and rho hold its first r.K weightings
// prepare_only: set up the solve's tables, state, plans and maps and return
// before capturing its graph (a group solve, run_group, runs the iterations)
int run_solve(ResultData& r, const double* W, const double* rho, const double* q1_init,
              const double* q2_init, const uint32_t* mask, const StreamSpec* stream = nullptr,
              bool prepare_only = false);
// Group solve: G (<= 4) prepared batch solves of different cases on one
// device, every tensor-core GEMM of an iteration one launch over all of them
// (iter.cu).  Same iteration form, tolerance, iteration cap and residual-test
// spacing for all; each keeps its own control block and stops on its own.
int run_group(int G, ResultData* const* R);
int fetch_times(const ResultData& r, double* t, double* tau);
int fetch_doses(const ResultData& r, const double* phi_eval, int n_eval, double* dose);
int fetch_stats(const ResultData& r, int* iters, double* obj, double* rel_pri,
                double* rel_dual, uint8_t* converged);
int fetch_state(const ResultData& r, double* q1, double* q2);
int times_into(const ResultData& r, double* t_dev);   // K x n_beams FP64, device
int fetch_metrics(const ResultData& r, const double* phi_eval, int n_eval, const int* label,
                  double* coverage, double* selectivity, double* gi, double* bot);
// 0 when a result may be read (its asynchronous solve, if any, waited for)
int result_ready(ResultData& d);
// FP64 check of the listed live columns (check.cu): out [nc][LGK_CHECK_COUNT], host
int run_check(ResultData& r, const int* cols, int nc, double* out);
// FP64 check of nc saved state columns with their tables (check.cu)
int run_check_states(ResultData& r, const float* q1, const float* q2, int nc, const int* src, const int* mcol,
                     const float* uf, const float* rhof, const float* wbf, const double* u64,
                     const double* wb64, double* out);

// FP64 GEMM (setup.cu):  C = alpha op(A) op(B) + beta C, row-major.
int dgemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, double alpha,
          const double* A, int lda, const double* B, int ldb, double beta,
          double* C, int ldc);

// BF16 tensor map of `parts` stacked [rows][cols] matrices, box 64 x box_rows (tc_gemm.cu)
int make_tma_map(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint64_t parts,
                 uint32_t box_rows);
// S = I + A A^T from the case's BF16 terms on the tensor cores (syrk.cu)
int tc_syrk(CaseData& cs, double* S, int* err);

// Tensor-core GEMMs (tc_gemm.cu)
int build_plan(GemmPlan& P, int rows, int col_tiles, int kb_total, int n_tile, bool split_first, int mt,
               int max_seg = 0);    // max_seg > 0: no segment crosses a multiple of max_seg k blocks
struct IterCtx;
int tc_check_product(CaseData& cs, bool transpose, const CUtensorMap& mA, const CUtensorMap& mB,
                     const GemmPlan& P, const IterCtx& cx, float* part, cudaStream_t st);
int sm_count();
struct IterCtx;
IterCtx make_ctx_public(ResultData& r);
int tc_prepare(ResultData& r);  // attributes + TMA maps, before capture
int tc_gemm1(ResultData& r, bool pdl = false);     // part[s] = Ahat . R1^T over split s of the columns
// c1 = A_lo . R1_hi^T, c2 = A_lo^T . V_hi^T (lo_refresh full iterations);
// first_only: skipped unless it is the solve's first iteration
int tc_gemm1_lo(ResultData& r, bool pdl = false, bool first_only = false);
int tc_gemm2_lo(ResultData& r, bool pdl = false, bool first_only = false);
int tc_solve(ResultData& r, bool pdl = false);     // part[s] = G3 . rhs^T  (6 products)
int tc_sv(ResultData& r, bool pdl = false);        // part[s] = S3 . V3^T   (6 products, refinement)
int tc_gemm2(ResultData& r, bool pdl = false);     // fused: q1, R1 update from Ahat^T . V
// the same products over a group of solves, one launch each, on stream st
int tc_group_gemm1(int G, ResultData* const* R, cudaStream_t st, bool pdl);
int tc_group_gemm1_lo(int G, ResultData* const* R, cudaStream_t st, bool pdl, bool first_only);
int tc_group_solve(int G, ResultData* const* R, cudaStream_t st, bool pdl);
int tc_group_sv(int G, ResultData* const* R, cudaStream_t st, bool pdl);
int tc_group_gemm2_lo(int G, ResultData* const* R, cudaStream_t st, bool pdl, bool first_only);
int tc_group_gemm2(int G, ResultData* const* R, cudaStream_t st, bool pdl);

}  // namespace lgk
