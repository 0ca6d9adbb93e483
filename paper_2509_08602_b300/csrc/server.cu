// Serving loop: planning requests (case + K weightings) admitted first come,
// first served under a device-memory budget, each run on a worker thread with
// its own CUDA stream so that requests in flight overlap on the device.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lgk_impl.hpp"

namespace lgk {

using Clock = std::chrono::steady_clock;

static double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    long long id = 0;
    // owned copies of the case description
    int n_iso = 0, n_pts = 0, n_targets = 0, n_oars = 0;
    double d_ld1 = 0, d_ld2 = 0, phi_cal = 0;
    std::vector<double> phi, d_presc, q_area, q_vol, d_oar, W;
    std::vector<uint8_t> kind;
    std::vector<uint16_t> sid;
    int K = 0;
    size_t footprint = 0;
    Clock::time_point t_submit, t_start, t_done;
    bool finished = false;
    lgk_request_info info{};
    std::string err;                 // error message of a failed request (worker's thread)
    std::vector<double> t, tau;

    lgk_case_desc desc() const {
        lgk_case_desc d{};
        d.n_iso = n_iso;
        d.n_pts = n_pts;
        d.n_targets = n_targets;
        d.n_oars = n_oars;
        d.phi = phi.data();
        d.kind = kind.data();
        d.struct_id = sid.data();
        d.d_presc = d_presc.data();
        d.q_area = q_area.data();
        d.q_vol = q_vol.data();
        d.d_oar = n_oars ? d_oar.data() : nullptr;
        d.d_ld1 = d_ld1;
        d.d_ld2 = d_ld2;
        d.phi_cal = phi_cal;
        return d;
    }
};

// Estimated peak device bytes of one request: the resident case (A terms,
// S^{-1} terms), the largest set-up temporaries (A in FP64, phi, S and
// L^{-1} in FP64) and the solve's state and scratch.
size_t request_footprint(int n_iso, int n_pts, int K, int precision) {
    const size_t B = 24ull * n_iso, m = B + n_iso, n = (size_t)n_pts + 8ull * n_iso;
    const size_t mp = (size_t)round_up((long long)m, 256), np = (size_t)round_up((long long)n, 256);
    const size_t a_res = precision == LGK_PREC_FP32 ? 4 * mp * np : (precision == LGK_PREC_BF16 ? 2 : 4) * mp * np;
    const size_t g_res = precision == LGK_PREC_FP32 ? 4 * mp * mp : 6 * mp * mp;
    const size_t setup = std::max<size_t>({8 * mp * np + 8 * (size_t)n_pts * B, 8 * mp * np + 8 * mp * mp,
                                           16 * mp * mp});
    const size_t Kp = (size_t)round_up(K, 32);
    const size_t solve = Kp * (12 * np + 22 * mp) + 4 * Kp * 128 * (size_t)(2 * 148 + np / 128 + 8) + (64u << 20);
    return a_res + g_res + setup + solve;
}

struct Server {
    lgk_server_params p{};
    int device = 0;
    size_t budget = 0, in_use = 0;
    bool stop = false;
    long long next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<long long, std::unique_ptr<Request>> reqs;
    std::vector<cudaStream_t> streams;
    std::vector<std::thread> workers;

    void run(Request& q, cudaStream_t st) {
        lgk_params prm = p.case_params;
        prm.stream = st;
        lgk_case_desc d = q.desc();
        lgk_case* cs = nullptr;
        lgk_result* res = nullptr;
        int rc = lgk_create_case(&d, &prm, &cs);
        const auto t_setup = Clock::now();
        q.info.setup_ms = ms_between(q.t_start, t_setup);
        if (rc == LGK_OK) {
            double beta = 1.0;
            lgk_case_info(cs, nullptr, nullptr, &beta, nullptr);
            rc = lgk_solve_weightings(cs, q.K, q.W.data(), nullptr, p.w0_bot, p.rho0_per_beta * beta,
                                      p.tol, p.max_iter, &res);
        }
        if (rc == LGK_OK) {
            q.t.resize((size_t)q.K * 24 * q.n_iso);
            q.tau.resize((size_t)q.K * q.n_iso);
            rc = lgk_fetch_times(res, q.t.data(), q.tau.data());
        }
        if (rc == LGK_OK) {
            std::vector<int> it(q.K);
            std::vector<uint8_t> conv(q.K);
            rc = lgk_fetch_stats(res, it.data(), nullptr, nullptr, nullptr, conv.data());
            for (int j = 0; j < q.K; ++j) {
                q.info.max_iters = std::max(q.info.max_iters, it[j]);
                q.info.converged += conv[j];
            }
        }
        q.info.solve_ms = ms_between(t_setup, Clock::now());
        if (rc != LGK_OK) q.err = lgk_last_error();
        lgk_free_result(res);
        lgk_destroy_case(cs);
        q.info.status = rc;
    }

    void worker(int w) {
        cudaSetDevice(device);
        for (;;) {
            Request* q = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] {
                    return stop || (!queue.empty() && in_use + queue.front()->footprint <= budget);
                });
                if (stop) return;
                q = queue.front();
                queue.pop_front();
                in_use += q->footprint;
                q->t_start = Clock::now();
            }
            try {
                run(*q, streams[w]);
            } catch (const std::exception& e) {
                set_error(std::string("server worker: ") + e.what());
                q->info.status = LGK_ECUDA;
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                in_use -= q->footprint;
                q->t_done = Clock::now();
                q->info.queue_ms = ms_between(q->t_submit, q->t_start);
                q->info.total_ms = ms_between(q->t_submit, q->t_done);
                q->finished = true;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }
};

}  // namespace lgk

struct lgk_server {
    lgk::Server s;
};

using namespace lgk;

extern "C" {

int lgk_server_create(const lgk_server_params* p, lgk_server** out) {
    if (!out || !p) {
        set_error("lgk_server_create: NULL argument");
        return LGK_EINVAL;
    }
    *out = nullptr;
    if (p->workers < 1 || p->workers > 64 || p->max_iter < 1 || !(p->tol >= 0) || !(p->w0_bot > 0) ||
        !(p->rho0_per_beta > 0)) {
        set_error("lgk_server_create: need 1 <= workers <= 64, max_iter >= 1, tol >= 0, w0_bot > 0, "
                  "rho0_per_beta > 0");
        return LGK_EINVAL;
    }
    std::unique_ptr<lgk_server> h(new (std::nothrow) lgk_server);
    if (!h) {
        set_error("host allocation failed");
        return LGK_ENOMEM;
    }
    Server& s = h->s;
    s.p = *p;
    s.device = p->case_params.device;
    LGK_CUDA_TRY(cudaSetDevice(s.device));
    s.budget = p->hbm_budget;
    if (!s.budget) {
        size_t fr = 0, tot = 0;
        LGK_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        s.budget = (size_t)(0.9 * (double)fr);
    }
    s.streams.resize(p->workers);
    for (auto& st : s.streams) LGK_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (int w = 0; w < p->workers; ++w) s.workers.emplace_back(&Server::worker, &s, w);
    *out = h.release();
    return LGK_OK;
}

int lgk_server_submit(lgk_server* h, const lgk_case_desc* d, int K, const double* W, long long* id) {
    if (!h || !d || !W || !id || K < 1 || K > 4096 || !d->phi || !d->kind || !d->struct_id ||
        !d->d_presc || !d->q_area || !d->q_vol || d->n_iso < 1 || d->n_pts < 1 || d->n_targets < 1 ||
        d->n_oars < 0 || (d->n_oars > 0 && !d->d_oar)) {
        set_error("lgk_server_submit: invalid argument");
        return LGK_EINVAL;
    }
    Server& s = h->s;
    auto q = std::make_unique<Request>();
    q->t_submit = Clock::now();
    q->n_iso = d->n_iso;
    q->n_pts = d->n_pts;
    q->n_targets = d->n_targets;
    q->n_oars = d->n_oars;
    q->d_ld1 = d->d_ld1;
    q->d_ld2 = d->d_ld2;
    q->phi_cal = d->phi_cal;
    const size_t B = 24ull * d->n_iso;
    q->phi.assign(d->phi, d->phi + (size_t)d->n_pts * B);
    q->kind.assign(d->kind, d->kind + d->n_pts);
    q->sid.assign(d->struct_id, d->struct_id + d->n_pts);
    q->d_presc.assign(d->d_presc, d->d_presc + d->n_targets);
    q->q_area.assign(d->q_area, d->q_area + d->n_targets);
    q->q_vol.assign(d->q_vol, d->q_vol + d->n_targets);
    if (d->n_oars) q->d_oar.assign(d->d_oar, d->d_oar + d->n_oars);
    q->W.assign(W, W + (size_t)K * 4);
    q->K = K;
    q->info.K = K;
    q->info.n_iso = d->n_iso;
    q->footprint = request_footprint(d->n_iso, d->n_pts, K, s.p.case_params.precision);
    q->info.footprint = q->footprint;
    if (q->footprint > s.budget) {
        set_error("lgk_server_submit: request needs ~" + std::to_string(q->footprint) +
                  " device bytes, more than the server budget of " + std::to_string(s.budget));
        return LGK_EBUDGET;
    }
    {
        std::lock_guard<std::mutex> lk(s.mu);
        q->id = s.next_id++;
        *id = q->id;
        s.queue.push_back(q.get());
        s.reqs[q->id] = std::move(q);
    }
    s.cv_work.notify_all();
    return LGK_OK;
}

int lgk_server_wait(lgk_server* h, long long id, int timeout_ms, lgk_request_info* info, double* t,
                    double* tau) {
    if (!h) {
        set_error("lgk_server_wait: server is NULL");
        return LGK_EINVAL;
    }
    Server& s = h->s;
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.reqs.find(id);
    if (it == s.reqs.end()) {
        set_error("lgk_server_wait: unknown request id (or already collected)");
        return LGK_EINVAL;
    }
    Request* q = it->second.get();
    if (!s.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return q->finished; })) {
        set_error("lgk_server_wait: request not finished within timeout_ms");
        return LGK_ETIMEOUT;
    }
    if (info) *info = q->info;
    if (t && !q->t.empty()) std::copy(q->t.begin(), q->t.end(), t);
    if (tau && !q->tau.empty()) std::copy(q->tau.begin(), q->tau.end(), tau);
    const int status = q->info.status;
    if (status != LGK_OK) set_error("request " + std::to_string(id) + ": " + q->err);
    s.reqs.erase(it);
    return status;
}

void lgk_server_destroy(lgk_server* h) {
    if (!h) return;
    Server& s = h->s;
    {
        std::lock_guard<std::mutex> lk(s.mu);
        s.stop = true;
        s.queue.clear();
    }
    s.cv_work.notify_all();
    for (auto& w : s.workers) w.join();
    for (auto& st : s.streams) cudaStreamDestroy(st);
    delete h;
}

}  // extern "C"
