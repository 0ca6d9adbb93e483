// C ABI of liblgk: argument checking, handle ownership, error reporting.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "lgk_impl.hpp"

struct lgk_case {
    std::shared_ptr<lgk::CaseData> d;
};
struct lgk_result {
    std::unique_ptr<lgk::ResultData> d;
};

namespace lgk {

static thread_local std::string g_err;
static thread_local long long g_launches = 0;

void set_error(const std::string& msg) { g_err = msg; }
void count_launch(long long n) { g_launches += n; }

CaseData::~CaseData() {
    if (stream) cudaStreamSynchronize(stream);
    if (cublas) cublasDestroy(cublas);
    if (own_stream && stream) cudaStreamDestroy(stream);
}

static int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

static bool finite_nonneg(const double* a, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!(a[i] >= 0.0) || !isfinite(a[i])) return false;
    return true;
}

static bool finite_pos(const double* a, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!(a[i] > 0.0) || !isfinite(a[i])) return false;
    return true;
}

// A result's solve has finished and, if it ran asynchronously, lgk_wait has
// reported its success: its results may be read.
int result_ready(ResultData& d) {
    std::lock_guard<std::mutex> lk(d.amu);
    if (!d.waited) return fail(LGK_EINVAL, "asynchronous solve not waited for: call lgk_wait first");
    if (d.async_rc) return fail(LGK_EINVAL, "the asynchronous solve of this result failed");
    return LGK_OK;
}

}  // namespace lgk

using namespace lgk;

extern "C" {

int lgk_default_params(lgk_params* p) {
    if (!p) return fail(LGK_EINVAL, "lgk_default_params: p is NULL");
    p->precision = LGK_PREC_BF16X3;
    p->normalize_rows = 1;
    p->scale_bot = 1;
    p->check_every = 10;
    p->eps_abs = 1e-12;
    p->device = 0;
    p->stream = nullptr;
    p->hbm_budget = 0;
    p->timeout_ms = 600000;
    p->profile = 0;
    p->lo_refresh = 1;
    p->lo_refresh_iters = 8000;
    p->rho_adapt = 0;
    p->solve_refine = 0;
    p->setup_fp64 = 0;
    p->check_fp64 = 0;
    p->autotune = 0;
    p->refine_after = 4000;
    p->l2_keep_inverse = 0;
    p->gemm2_tile_rows = 0;
    p->accum_kblocks = 64;
    return LGK_OK;
}

int lgk_create_case(const lgk_case_desc* d, const lgk_params* p, lgk_case** out) {
    if (!out) return fail(LGK_EINVAL, "lgk_create_case: out is NULL");
    *out = nullptr;
    if (!d) return fail(LGK_EINVAL, "lgk_create_case: desc is NULL");
    lgk_params prm;
    lgk_default_params(&prm);
    if (p) prm = *p;
    if (prm.lo_refresh != 0 && prm.lo_refresh != 1) return fail(LGK_EINVAL, "lo_refresh must be 0 or 1");
    if (prm.lo_refresh_iters < 0) return fail(LGK_EINVAL, "lo_refresh_iters must be >= 0");
    if (prm.rho_adapt != 0 && prm.rho_adapt != 1) return fail(LGK_EINVAL, "rho_adapt must be 0 or 1");
    if (prm.solve_refine < 0 || prm.solve_refine > 2) return fail(LGK_EINVAL, "solve_refine must be 0, 1 or 2");
    if (prm.setup_fp64 != 0 && prm.setup_fp64 != 1) return fail(LGK_EINVAL, "setup_fp64 must be 0 or 1");
    if (prm.check_fp64 != 0 && prm.check_fp64 != 1) return fail(LGK_EINVAL, "check_fp64 must be 0 or 1");
    if (prm.autotune != 0 && prm.autotune != 1) return fail(LGK_EINVAL, "autotune must be 0 or 1");
    if (prm.refine_after < 0) return fail(LGK_EINVAL, "refine_after must be >= 0");
    if (prm.l2_keep_inverse != 0 && prm.l2_keep_inverse != 1)
        return fail(LGK_EINVAL, "l2_keep_inverse must be 0 or 1");
    if (prm.gemm2_tile_rows != 0 && prm.gemm2_tile_rows != 128 && prm.gemm2_tile_rows != 256)
        return fail(LGK_EINVAL, "gemm2_tile_rows must be 0, 128 or 256");
    if (prm.accum_kblocks < 0) return fail(LGK_EINVAL, "accum_kblocks must be >= 0");
    if (prm.precision != LGK_PREC_FP32 && prm.precision != LGK_PREC_BF16 &&
        prm.precision != LGK_PREC_BF16X3)
        return fail(LGK_EINVAL, "unknown precision");
    if (prm.check_every < 1 || !(prm.eps_abs >= 0.0) || prm.timeout_ms < 1)
        return fail(LGK_EINVAL, "check_every >= 1, eps_abs >= 0 and timeout_ms >= 1 required");
    if (d->n_iso < 1 || d->n_pts < 1 || d->n_targets < 1 || d->n_targets > kMaxTargets || d->n_oars < 0)
        return fail(LGK_EINVAL, "need n_iso >= 1, n_pts >= 1, 1 <= n_targets <= 64, n_oars >= 0");
    const long long B = 24LL * d->n_iso, m = B + d->n_iso, n = (long long)d->n_pts + 8LL * d->n_iso;
    if (round_up(m, 128) * round_up(n, 128) >= (1LL << 40) || n >= (1LL << 30))
        return fail(LGK_EINVAL, "problem too large");
    if (!d->phi || !d->kind || !d->struct_id || !d->d_presc || !d->q_area || !d->q_vol ||
        (d->n_oars > 0 && !d->d_oar))
        return fail(LGK_EINVAL, "NULL input array");
    if (!finite_pos(d->d_presc, d->n_targets) || !finite_nonneg(d->q_area, d->n_targets) ||
        !finite_nonneg(d->q_vol, d->n_targets) || (d->n_oars && !finite_pos(d->d_oar, d->n_oars)) ||
        !(d->d_ld1 > 0) || !(d->d_ld2 > 0) || !(d->phi_cal > 0) || !isfinite(d->d_ld1) ||
        !isfinite(d->d_ld2) || !isfinite(d->phi_cal))
        return fail(LGK_EINVAL, "thresholds must be finite and > 0, q shares finite and >= 0");
    for (int i = 0; i < d->n_pts; ++i) {
        int k = d->kind[i], s = d->struct_id[i];
        if (k > LGK_OAR) return fail(LGK_EINVAL, "point " + std::to_string(i) + ": unknown class");
        if (k <= LGK_R && s >= d->n_targets)
            return fail(LGK_EINVAL, "point " + std::to_string(i) + ": target index out of range");
        if (k == LGK_OAR && s >= d->n_oars)
            return fail(LGK_EINVAL, "point " + std::to_string(i) + ": OAR index out of range");
    }
    // phi (n_pts x 24 n_iso, up to GBs) is validated on the device as it is
    // assembled (setup_case): a host scan here took longer than the set-up

    std::shared_ptr<CaseData> cs;
    try {
        cs = std::make_shared<CaseData>();
    } catch (const std::bad_alloc&) {
        return fail(LGK_ENOMEM, "host allocation failed");
    }
    cs->prm = prm;
    cs->device = prm.device;
    LGK_CUDA_TRY(cudaSetDevice(prm.device));
    if (prm.stream) {
        cs->stream = static_cast<cudaStream_t>(prm.stream);
    } else {
        LGK_CUDA_TRY(cudaStreamCreateWithFlags(&cs->stream, cudaStreamNonBlocking));
        cs->own_stream = true;
    }
    if (prm.precision == LGK_PREC_FP32) {
        if (cublasCreate(&cs->cublas) != CUBLAS_STATUS_SUCCESS) return fail(LGK_ECUDA, "cublasCreate failed");
        cublasSetMathMode(cs->cublas, CUBLAS_PEDANTIC_MATH);     // strict FP32, no TF32
        cublasSetStream(cs->cublas, cs->stream);
        int rc = cs->cublas_ws.alloc(32u << 20);
        if (rc) return rc;
        cublasSetWorkspace(cs->cublas, cs->cublas_ws.p, cs->cublas_ws.bytes);
    }
    int rc;
    try {
        rc = setup_case(*cs, *d);
    } catch (const std::bad_alloc&) {
        rc = fail(LGK_ENOMEM, "host allocation failed");
    }
    if (rc) return rc;
    lgk_case* h = new (std::nothrow) lgk_case;
    if (!h) return fail(LGK_ENOMEM, "host allocation failed");
    h->d = std::move(cs);
    *out = h;
    return LGK_OK;
}

int lgk_case_info(const lgk_case* c, int* m, int* n, double* beta, size_t* bytes) {
    if (!c) return fail(LGK_EINVAL, "case is NULL");
    if (m) *m = c->d->m;
    if (n) *n = c->d->n;
    if (beta) *beta = c->d->beta;
    if (bytes) *bytes = c->d->bytes_held();
    return LGK_OK;
}

// Per-weighting penalties: the caller's, or Eq. rho_rule.
static int column_rho(int K, const double* W, const double* rho, double w0_bot, double rho0,
                      std::vector<double>& r) {
    r.assign(K, 0.0);
    if (rho) {
        if (!finite_pos(rho, K)) return fail(LGK_EINVAL, "rho must be finite and > 0");
        r.assign(rho, rho + K);
        return LGK_OK;
    }
    if (!(w0_bot > 0) || !(rho0 > 0) || !isfinite(w0_bot) || !isfinite(rho0))
        return fail(LGK_EINVAL, "rho rule needs w0_bot > 0 and rho0 > 0");
    for (int j = 0; j < K; ++j) {
        if (!(W[4 * (size_t)j + 3] > 0)) return fail(LGK_EINVAL, "rho rule needs w_BOT > 0");
        r[j] = rho0 * sqrt(w0_bot / W[4 * (size_t)j + 3]);     // Eq. rho_rule
    }
    return LGK_OK;
}

static int ready(const lgk_result* r) {
    if (!r) return fail(LGK_EINVAL, "result is NULL");
    return result_ready(*r->d);
}

static int case_free(const lgk_case* c) {
    if (c->d->async_busy.load())
        return fail(LGK_EINVAL, "case busy: an asynchronous solve of it is running (lgk_wait first)");
    return LGK_OK;
}

int lgk_solve_weightings_masked(lgk_case* c, int K, const double* W, const double* rho, double w0_bot,
                                double rho0, double tol, int max_iter, const uint32_t* mask,
                                const double* q1_init, const double* q2_init, lgk_result** out) {
    if (!out) return fail(LGK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!c || !W) return fail(LGK_EINVAL, "case or W is NULL");
    if (int rb = case_free(c)) return rb;
    if (K < 1 || K > 4096) return fail(LGK_EINVAL, "need 1 <= K <= 4096");
    if (!finite_nonneg(W, (size_t)K * 4)) return fail(LGK_EINVAL, "weights must be finite and >= 0");
    if (!(tol >= 0.0) || !isfinite(tol) || max_iter < 1) return fail(LGK_EINVAL, "need tol >= 0, max_iter >= 1");
    std::vector<double> r;
    int rrc = column_rho(K, W, rho, w0_bot, rho0, r);
    if (rrc) return rrc;
    LGK_CUDA_TRY(cudaSetDevice(c->d->device));
    std::unique_ptr<ResultData> res;
    try {
        res.reset(new ResultData);
    } catch (const std::bad_alloc&) {
        return fail(LGK_ENOMEM, "host allocation failed");
    }
    res->cs = c->d;
    res->K = K;
    res->tol = tol;
    res->max_iter = max_iter;
    if ((q1_init && !std::all_of(q1_init, q1_init + (size_t)K * c->d->n, [](double v) { return isfinite(v); })) ||
        (q2_init && !std::all_of(q2_init, q2_init + (size_t)K * c->d->m, [](double v) { return isfinite(v); })))
        return fail(LGK_EINVAL, "initial state must be finite");
    int rc;
    try {
        rc = run_solve(*res, W, r.data(), q1_init, q2_init, mask);
    } catch (const std::bad_alloc&) {
        rc = fail(LGK_ENOMEM, "host allocation failed");
    }
    if (rc) return rc;
    lgk_result* h = new (std::nothrow) lgk_result;
    if (!h) return fail(LGK_ENOMEM, "host allocation failed");
    h->d = std::move(res);
    *out = h;
    return LGK_OK;
}

int lgk_solve_group(int G, lgk_case* const* cases, const int* K, const double* const* W,
                    const double* const* rho, double w0_bot, const double* rho0, double tol, int max_iter,
                    lgk_result** out) {
    if (!out) return fail(LGK_EINVAL, "out is NULL");
    if (G < 1 || G > 4) return fail(LGK_EINVAL, "need 1 <= G <= 4");
    for (int g = 0; g < G; ++g) out[g] = nullptr;
    if (!cases || !K || !W) return fail(LGK_EINVAL, "cases, K or W is NULL");
    if (!(tol >= 0.0) || !isfinite(tol) || max_iter < 1) return fail(LGK_EINVAL, "need tol >= 0, max_iter >= 1");
    std::vector<std::vector<double>> rr(G);
    for (int g = 0; g < G; ++g) {
        if (!cases[g] || !W[g]) return fail(LGK_EINVAL, "a case or its W is NULL");
        for (int h = 0; h < g; ++h)
            if (cases[h] == cases[g]) return fail(LGK_EINVAL, "a case appears twice in the group");
        if (int rb = case_free(cases[g])) return rb;
        if (K[g] < 1 || K[g] > 4096) return fail(LGK_EINVAL, "need 1 <= K <= 4096 per case");
        if (!finite_nonneg(W[g], (size_t)K[g] * 4)) return fail(LGK_EINVAL, "weights must be finite and >= 0");
        int rrc = column_rho(K[g], W[g], rho ? rho[g] : nullptr, w0_bot, rho0 ? rho0[g] : 0.0, rr[g]);
        if (rrc) return rrc;
    }
    LGK_CUDA_TRY(cudaSetDevice(cases[0]->d->device));
    std::vector<std::unique_ptr<ResultData>> res(G);
    std::vector<ResultData*> raw(G);
    int rc = LGK_OK;
    try {
        for (int g = 0; g < G && !rc; ++g) {
            res[g].reset(new ResultData);
            res[g]->cs = cases[g]->d;
            res[g]->K = K[g];
            res[g]->tol = tol;
            res[g]->max_iter = max_iter;
            raw[g] = res[g].get();
            if (cases[g]->d->device != cases[0]->d->device)
                rc = fail(LGK_EINVAL, "a group's cases must share one device");
            else
                rc = run_solve(*res[g], W[g], rr[g].data(), nullptr, nullptr, nullptr, nullptr, true);
        }
        if (!rc) rc = run_group(G, raw.data());
    } catch (const std::bad_alloc&) {
        rc = fail(LGK_ENOMEM, "host allocation failed");
    }
    if (rc) return rc;
    std::vector<lgk_result*> hs(G, nullptr);
    for (int g = 0; g < G; ++g) {
        hs[g] = new (std::nothrow) lgk_result;
        if (!hs[g]) {
            for (int h = 0; h < g; ++h) delete hs[h];
            return fail(LGK_ENOMEM, "host allocation failed");
        }
    }
    for (int g = 0; g < G; ++g) {
        hs[g]->d = std::move(res[g]);
        out[g] = hs[g];
    }
    return LGK_OK;
}

int lgk_solve_weightings_warm(lgk_case* c, int K, const double* W, const double* rho, double w0_bot,
                              double rho0, double tol, int max_iter, const double* q1_init,
                              const double* q2_init, lgk_result** out) {
    return lgk_solve_weightings_masked(c, K, W, rho, w0_bot, rho0, tol, max_iter, nullptr, q1_init,
                                       q2_init, out);
}

int lgk_solve_weightings(lgk_case* c, int K, const double* W, const double* rho, double w0_bot,
                         double rho0, double tol, int max_iter, lgk_result** out) {
    return lgk_solve_weightings_masked(c, K, W, rho, w0_bot, rho0, tol, max_iter, nullptr, nullptr,
                                       nullptr, out);
}

int lgk_solve_weightings_async(lgk_case* c, int K, const double* W, const double* rho, double w0_bot,
                               double rho0, double tol, int max_iter, lgk_result** out) {
    if (!out) return fail(LGK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!c || !W) return fail(LGK_EINVAL, "case or W is NULL");
    if (K < 1 || K > 4096) return fail(LGK_EINVAL, "need 1 <= K <= 4096");
    if (!finite_nonneg(W, (size_t)K * 4)) return fail(LGK_EINVAL, "weights must be finite and >= 0");
    if (!(tol >= 0.0) || !isfinite(tol) || max_iter < 1) return fail(LGK_EINVAL, "need tol >= 0, max_iter >= 1");
    std::vector<double> r;
    int rrc = column_rho(K, W, rho, w0_bot, rho0, r);
    if (rrc) return rrc;
    int expect = 0;
    if (!c->d->async_busy.compare_exchange_strong(expect, 1))
        return fail(LGK_EINVAL, "case busy: an asynchronous solve of it is running (lgk_wait first)");
    lgk_result* h = nullptr;
    try {
        std::vector<double> w(W, W + (size_t)K * 4);
        std::unique_ptr<ResultData> res(new ResultData);
        res->cs = c->d;
        res->K = K;
        res->tol = tol;
        res->max_iter = max_iter;
        res->running = true;
        res->waited = false;
        h = new lgk_result;
        h->d = std::move(res);
        ResultData* rd = h->d.get();
        rd->worker = std::thread([rd, w = std::move(w), r = std::move(r)]() {
            int rc = LGK_OK;
            if (cudaSetDevice(rd->cs->device) != cudaSuccess) {
                cudaGetLastError();
                rc = fail(LGK_ECUDA, "cudaSetDevice failed in the solve thread");
            } else {
                try {
                    rc = run_solve(*rd, w.data(), r.data(), nullptr, nullptr, nullptr);
                } catch (const std::bad_alloc&) {
                    rc = fail(LGK_ENOMEM, "host allocation failed");
                }
            }
            rd->cs->async_busy = 0;
            std::lock_guard<std::mutex> lk(rd->amu);
            rd->async_rc = rc;
            rd->async_err = rc ? g_err : std::string();
            rd->running = false;
            rd->acv.notify_all();
        });
    } catch (const std::exception&) {     // bad_alloc, or std::system_error from std::thread
        c->d->async_busy = 0;
        delete h;
        return fail(LGK_ENOMEM, "could not start the solve thread");
    }
    *out = h;
    return LGK_OK;
}

int lgk_wait(lgk_result* r, int timeout_ms) {
    if (!r) return fail(LGK_EINVAL, "result is NULL");
    if (timeout_ms < 0) return fail(LGK_EINVAL, "timeout_ms must be >= 0");
    ResultData& d = *r->d;
    {
        std::unique_lock<std::mutex> lk(d.amu);
        if (!d.acv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !d.running; }))
            return fail(LGK_ETIMEOUT, "solve still running after timeout_ms");
    }
    if (d.worker.joinable()) d.worker.join();
    std::lock_guard<std::mutex> lk(d.amu);
    if (d.async_rc) return fail(d.async_rc, d.async_err);
    d.waited = true;
    return LGK_OK;
}

int lgk_solve_stream(lgk_case* c, int K_total, const double* W, const double* rho, double w0_bot,
                     double rho0, double tol, int max_iter, int width, double* t, double* tau, int* iters,
                     double* obj, double* rel_pri, double* rel_dual, uint8_t* converged, double* prof_ms,
                     long long* prof_launches, double* check) {
    if (!c || !W) return fail(LGK_EINVAL, "case or W is NULL");
    if (int rb = case_free(c)) return rb;
    if (K_total < 1 || K_total > (1 << 20) || width < 1 || width > 4096)
        return fail(LGK_EINVAL, "need 1 <= K_total <= 2^20 and 1 <= width <= 4096");
    if (!finite_nonneg(W, (size_t)K_total * 4)) return fail(LGK_EINVAL, "weights must be finite and >= 0");
    if (!(tol >= 0.0) || !isfinite(tol) || max_iter < 1) return fail(LGK_EINVAL, "need tol >= 0, max_iter >= 1");
    if ((prof_ms || prof_launches) && !c->d->prm.profile)
        return fail(LGK_EINVAL, "profile outputs need lgk_params.profile = 1");
    {
        // The stream's iteration counter is a 32-bit int on the device.  A
        // weighting holds its column for at most its cap rounded up to a graph
        // replay plus one replay, and every column stays busy until the queue
        // is empty, so the counter never passes
        // (ceil(K_total / width) + 1) x (round_up(max_iter, replay) + replay).
        const long long replay = 5LL * std::max(1, c->d->prm.check_every);
        const long long per_w = round_up(max_iter, replay) + replay;
        const long long rounds = (K_total + (long long)width - 1) / width + 1;
        if ((double)rounds * (double)per_w > (double)(1 << 30))
            return fail(LGK_EINVAL, "K_total / width x max_iter too large: the stream's iteration count "
                                    "could pass 2^30; lower max_iter or K_total, or raise width");
    }
    std::vector<double> r;
    int rc = column_rho(K_total, W, rho, w0_bot, rho0, r);
    if (rc) return rc;
    LGK_CUDA_TRY(cudaSetDevice(c->d->device));
    std::unique_ptr<ResultData> res;
    try {
        res.reset(new ResultData);
    } catch (const std::bad_alloc&) {
        return fail(LGK_ENOMEM, "host allocation failed");
    }
    res->cs = c->d;
    res->K = std::min(width, K_total);
    res->tol = tol;
    res->max_iter = 1 << 30;        // the device never stops a column on its count; the host does
    StreamSpec ss;
    ss.K_total = K_total;
    ss.W = W;
    ss.rho = r.data();
    ss.max_iter = max_iter;
    ss.t = t;
    ss.tau = tau;
    ss.iters = iters;
    ss.obj = obj;
    ss.rel_pri = rel_pri;
    ss.rel_dual = rel_dual;
    ss.converged = converged;
    ss.check = check;
    try {
        rc = run_solve(*res, W, r.data(), nullptr, nullptr, nullptr, &ss);
    } catch (const std::bad_alloc&) {
        rc = fail(LGK_ENOMEM, "host allocation failed");
    }
    if (rc) return rc;
    for (int k = 0; k < LGK_K_COUNT; ++k) {
        if (prof_ms) prof_ms[k] = res->prof_ms[k];
        if (prof_launches) prof_launches[k] = res->prof_n[k];
    }
    return LGK_OK;
}

int lgk_fetch_times(const lgk_result* r, double* t, double* tau) {
    if (int rb = ready(r)) return rb;
    LGK_CUDA_TRY(cudaSetDevice(r->d->cs->device));
    return fetch_times(*r->d, t, tau);
}

int lgk_fetch_doses(const lgk_result* r, const double* phi_eval, int n_eval, double* dose) {
    if (!r || !phi_eval || !dose || n_eval < 1) return fail(LGK_EINVAL, "bad fetch_doses arguments");
    if (!finite_nonneg(phi_eval, (size_t)n_eval * r->d->cs->n_beams))
        return fail(LGK_EINVAL, "phi_eval must be finite and >= 0");
    if (int rb = ready(r)) return rb;
    LGK_CUDA_TRY(cudaSetDevice(r->d->cs->device));
    return fetch_doses(*r->d, phi_eval, n_eval, dose);
}

int lgk_fetch_metrics(const lgk_result* r, const double* phi_eval, int n_eval, const int* label,
                      double* coverage, double* selectivity, double* gi, double* bot) {
    if (!r || !phi_eval || !label || n_eval < 1) return fail(LGK_EINVAL, "bad fetch_metrics arguments");
    if (int rb = ready(r)) return rb;
    const CaseData& cs = *r->d->cs;
    if (!finite_nonneg(phi_eval, (size_t)n_eval * cs.n_beams))
        return fail(LGK_EINVAL, "phi_eval must be finite and >= 0");
    for (int e = 0; e < n_eval; ++e)
        if (label[e] < -1 || label[e] >= cs.n_targets)
            return fail(LGK_EINVAL, "label " + std::to_string(e) + " out of range");
    LGK_CUDA_TRY(cudaSetDevice(cs.device));
    return fetch_metrics(*r->d, phi_eval, n_eval, label, coverage, selectivity, gi, bot);
}

int lgk_fetch_stats(const lgk_result* r, int* iters, double* obj, double* rel_pri, double* rel_dual,
                    uint8_t* converged) {
    if (int rb = ready(r)) return rb;
    LGK_CUDA_TRY(cudaSetDevice(r->d->cs->device));
    return fetch_stats(*r->d, iters, obj, rel_pri, rel_dual, converged);
}

int lgk_fetch_check(const lgk_result* r, double* out) {
    if (!r || !out) return fail(LGK_EINVAL, "result or out is NULL");
    if (int rb = ready(r)) return rb;
    LGK_CUDA_TRY(cudaSetDevice(r->d->cs->device));
    ResultData& rd = *r->d;
    if (rd.u64.empty()) return fail(LGK_EINVAL, "result holds no solve");
    std::vector<int> cols(rd.K);
    for (int j = 0; j < rd.K; ++j) cols[j] = j;
    try {
        return run_check(rd, cols.data(), rd.K, out);
    } catch (const std::bad_alloc&) {
        return fail(LGK_ENOMEM, "host allocation failed");
    }
}

int lgk_fetch_state(const lgk_result* r, double* q1, double* q2) {
    if (int rb = ready(r)) return rb;
    LGK_CUDA_TRY(cudaSetDevice(r->d->cs->device));
    return fetch_state(*r->d, q1, q2);
}

int lgk_fetch_profile(const lgk_result* r, double* ms, long long* launches) {
    if (int rb = ready(r)) return rb;
    if (!r->d->cs->prm.profile) return fail(LGK_EINVAL, "solve was not profiled (lgk_params.profile = 0)");
    for (int k = 0; k < LGK_K_COUNT; ++k) {
        if (ms) ms[k] = r->d->prof_ms[k];
        if (launches) launches[k] = r->d->prof_n[k];
    }
    return LGK_OK;
}

void lgk_free_result(lgk_result* r) {
    if (!r) return;
    cudaSetDevice(r->d->cs->device);
    delete r;
}

void lgk_destroy_case(lgk_case* c) {
    if (!c) return;
    cudaSetDevice(c->d->device);
    delete c;
}

const char* lgk_last_error(void) { return g_err.c_str(); }

long long lgk_launch_count(void) {
    long long n = g_launches;
    g_launches = 0;
    return n;
}

}  // extern "C"
