// Serving loop with continuous batching.
//
// A resident case is one planning case (its A, S^{-1} and ADMM state on the
// device) admitted first come, first served under a device-memory budget.  A
// worker thread sets it up on its own CUDA stream and runs one streaming
// solve on it (lgk_solve_stream's machinery with a dynamic source): the
// solve has `stream_width` weighting columns, and every weighting submitted
// for the case -- by any request, at any time while the case is resident --
// waits in the case's queue and takes the next column that frees up (at the
// next graph replay boundary).  Requests that arrive while the case is on the
// GPU therefore join its running batch instead of waiting for it to finish,
// and cases on different workers overlap on the device.  A weighting's result
// does not depend on what runs beside it: columns never interact, and every
// column starts the same way.
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

// the case handle of the C ABI (the same definition as in api.cu)
struct lgk_case {
    std::shared_ptr<lgk::CaseData> d;
};

namespace lgk {

using Clock = std::chrono::steady_clock;

static double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    long long id = 0, case_id = 0;
    int K = 0, remaining = 0, n_iso = 0;
    Clock::time_point t_submit, t_first, t_done;
    bool started = false, finished = false;
    lgk_request_info info{};
    std::string err;
    std::vector<double> t, tau;
};

struct Job {
    long long req = 0;
    int idx = 0;
    double w[4] = {0, 0, 0, 0};
};

struct Resident {
    long long id = 0;
    // owned copy of the case description
    int n_iso = 0, n_pts = 0, n_targets = 0, n_oars = 0;
    double d_ld1 = 0, d_ld2 = 0, phi_cal = 0;
    std::vector<double> phi, d_presc, q_area, q_vol, d_oar;
    std::vector<uint8_t> kind;
    std::vector<uint16_t> sid;
    size_t footprint = 0;
    std::deque<Job> pending;              // weightings waiting for a column
    std::map<long long, Job> running;     // stream tag -> weighting in a column
    long long next_tag = 0;
    bool closed = false;                  // no more weightings will be submitted
    bool set_up = false, finished = false;
    int status = LGK_OK;
    std::string err;
    double setup_ms = 0.0;
    double beta = 1.0;
    std::condition_variable cv;           // new weightings or closed

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

// Estimated peak device bytes of one resident case: the case (A terms,
// S^{-1} terms), the largest set-up temporaries (A in FP64, phi, S and
// L^{-1} in FP64) and a solve of K columns with its scratch.
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
    int device = 0, width = 32;
    size_t budget = 0, in_use = 0;
    bool stop = false;
    long long next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Resident*> queue;                          // cases waiting for admission
    std::map<long long, std::unique_ptr<Resident>> cases;
    std::map<long long, std::unique_ptr<Request>> reqs;
    std::vector<cudaStream_t> streams;
    std::vector<std::thread> workers;

    // a resident case ended (set-up failed, solve failed, or server stopped):
    // its queued and running weightings fail with `status`
    void fail_case(Resident& rc, int status, const std::string& err) {
        auto fail_job = [&](const Job& j) {
            auto it = reqs.find(j.req);
            if (it == reqs.end()) return;
            Request& q = *it->second;
            if (q.finished) return;
            q.info.status = status;
            q.err = err;
            q.finished = true;
            q.t_done = Clock::now();
            q.info.total_ms = ms_between(q.t_submit, q.t_done);
        };
        for (const Job& j : rc.pending) fail_job(j);
        for (const auto& kv : rc.running) fail_job(kv.second);
        rc.pending.clear();
        rc.running.clear();
        rc.status = status;
        rc.err = err;
    }

    // the stream's source: the next queued weighting of the case
    int pull(Resident& rc, double* w, double* rho, long long* tag, bool block) {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            if (stop) return -1;
            if (!rc.pending.empty()) {
                Job j = rc.pending.front();
                rc.pending.pop_front();
                std::copy(j.w, j.w + 4, w);
                *rho = p.rho0_per_beta * rc.beta * sqrt(p.w0_bot / j.w[3]);    // Eq. rho_rule
                *tag = rc.next_tag++;
                rc.running[*tag] = j;
                auto it = reqs.find(j.req);
                if (it != reqs.end() && !it->second->started) {
                    it->second->started = true;
                    it->second->t_first = Clock::now();
                }
                return 1;
            }
            if (rc.closed) return -1;
            if (!block) return 0;
            rc.cv.wait_for(lk, std::chrono::milliseconds(100));
        }
    }

    void done(Resident& rc, long long tag, const StreamOut& o) {
        std::lock_guard<std::mutex> lk(mu);
        auto jt = rc.running.find(tag);
        if (jt == rc.running.end()) return;
        const Job j = jt->second;
        rc.running.erase(jt);
        auto it = reqs.find(j.req);
        if (it == reqs.end()) return;
        Request& q = *it->second;
        const size_t B = 24ull * rc.n_iso;
        std::copy(o.t, o.t + B, q.t.begin() + (size_t)j.idx * B);
        std::copy(o.tau, o.tau + rc.n_iso, q.tau.begin() + (size_t)j.idx * rc.n_iso);
        q.info.max_iters = std::max(q.info.max_iters, o.iters);
        q.info.converged += o.converged ? 1 : 0;
        if (--q.remaining == 0) {
            q.finished = true;
            q.t_done = Clock::now();
            q.info.status = LGK_OK;
            q.info.queue_ms = ms_between(q.t_submit, q.t_first);
            q.info.solve_ms = ms_between(q.t_first, q.t_done);
            q.info.total_ms = ms_between(q.t_submit, q.t_done);
            cv_done.notify_all();
        }
    }

    void run(Resident& rc, cudaStream_t st) {
        lgk_params prm = p.case_params;
        prm.stream = st;
        lgk_case_desc d = rc.desc();
        lgk_case* cs = nullptr;
        const auto t0 = Clock::now();
        int status = lgk_create_case(&d, &prm, &cs);
        std::string err = status ? std::string(lgk_last_error()) : std::string();
        {
            std::lock_guard<std::mutex> lk(mu);
            rc.setup_ms = ms_between(t0, Clock::now());
            rc.set_up = true;
            if (status == LGK_OK) lgk_case_info(cs, nullptr, nullptr, &rc.beta, nullptr);
            for (auto& kv : reqs)
                if (kv.second->case_id == rc.id && !kv.second->finished) kv.second->info.setup_ms = rc.setup_ms;
        }
        if (status == LGK_OK) {
            // the first weightings (wait for at least one, or for the case to close)
            std::vector<double> W((size_t)width * 4, 0.0), rho(width, 1.0);
            std::vector<long long> tags(width, -1);
            int n0 = 0;
            for (int j = 0; j < width; ++j) {
                if (pull(rc, &W[4 * (size_t)j], &rho[j], &tags[j], j == 0) != 1) break;
                ++n0;
            }
            if (n0 > 0) {
                StreamSpec ss;
                ss.max_iter = p.max_iter;
                ss.pull = [&](double* w, double* rh, long long* tag, bool block) {
                    return pull(rc, w, rh, tag, block);
                };
                ss.done = [&](long long tag, const StreamOut& o) { done(rc, tag, o); };
                ss.n_initial = n0;
                ss.initial_tags = tags.data();
                ResultData res;
                res.cs = cs->d;
                res.K = width;
                res.tol = p.tol;
                res.max_iter = 1 << 30;      // the host stops each column at its own cap
                try {
                    status = run_solve(res, W.data(), rho.data(), nullptr, nullptr, nullptr, &ss);
                } catch (const std::bad_alloc&) {
                    set_error("host allocation failed");
                    status = LGK_ENOMEM;
                }
                if (status) err = lgk_last_error();
            }
        }
        lgk_destroy_case(cs);
        std::lock_guard<std::mutex> lk(mu);
        if (status != LGK_OK || stop) fail_case(rc, status ? status : LGK_ETIMEOUT,
                                                status ? err : "server destroyed");
        rc.finished = true;
        cv_done.notify_all();
    }

    void worker(int w) {
        cudaSetDevice(device);
        for (;;) {
            Resident* rc = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] {
                    return stop || (!queue.empty() && in_use + queue.front()->footprint <= budget);
                });
                if (stop) return;
                rc = queue.front();
                queue.pop_front();
                in_use += rc->footprint;
            }
            try {
                run(*rc, streams[w]);
            } catch (const std::exception& e) {
                std::lock_guard<std::mutex> lk(mu);
                fail_case(*rc, LGK_ECUDA, std::string("server worker: ") + e.what());
                rc->finished = true;
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                in_use -= rc->footprint;
                cases.erase(rc->id);
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }

    // queue K weightings of resident case `rc` as request *id (lock held)
    void add_request(Resident& rc, int K, const double* W, long long* id) {
        auto q = std::make_unique<Request>();
        q->t_submit = Clock::now();
        q->id = next_id++;
        q->case_id = rc.id;
        q->K = q->remaining = K;
        q->n_iso = rc.n_iso;
        q->info.K = K;
        q->info.n_iso = rc.n_iso;
        q->info.footprint = rc.footprint;
        q->info.setup_ms = 0.0;       // set to the case's set-up time if it is still to come
        q->t.assign((size_t)K * 24 * rc.n_iso, 0.0);
        q->tau.assign((size_t)K * rc.n_iso, 0.0);
        for (int j = 0; j < K; ++j) {
            Job jb;
            jb.req = q->id;
            jb.idx = j;
            std::copy(W + 4 * (size_t)j, W + 4 * (size_t)j + 4, jb.w);
            rc.pending.push_back(jb);
        }
        *id = q->id;
        reqs[q->id] = std::move(q);
        rc.cv.notify_all();
    }
};

static bool valid_weights(int K, const double* W) {
    for (size_t i = 0; i < (size_t)K * 4; ++i)
        if (!(W[i] >= 0.0) || !isfinite(W[i])) return false;
    for (int j = 0; j < K; ++j)
        if (!(W[4 * (size_t)j + 3] > 0.0)) return false;      // the rho rule divides by w_BOT
    return true;
}

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
        !(p->rho0_per_beta > 0) || p->stream_width < 0 || p->stream_width > 4096) {
        set_error("lgk_server_create: need 1 <= workers <= 64, max_iter >= 1, tol >= 0, w0_bot > 0, "
                  "rho0_per_beta > 0, 0 <= stream_width <= 4096");
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
    s.width = p->stream_width ? p->stream_width : 32;
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

int lgk_server_open(lgk_server* h, const lgk_case_desc* d, long long* case_id) {
    if (!h || !d || !case_id || !d->phi || !d->kind || !d->struct_id || !d->d_presc || !d->q_area ||
        !d->q_vol || d->n_iso < 1 || d->n_pts < 1 || d->n_targets < 1 || d->n_oars < 0 ||
        (d->n_oars > 0 && !d->d_oar)) {
        set_error("lgk_server_open: invalid argument");
        return LGK_EINVAL;
    }
    Server& s = h->s;
    auto rc = std::make_unique<Resident>();
    rc->n_iso = d->n_iso;
    rc->n_pts = d->n_pts;
    rc->n_targets = d->n_targets;
    rc->n_oars = d->n_oars;
    rc->d_ld1 = d->d_ld1;
    rc->d_ld2 = d->d_ld2;
    rc->phi_cal = d->phi_cal;
    const size_t B = 24ull * d->n_iso;
    rc->phi.assign(d->phi, d->phi + (size_t)d->n_pts * B);
    rc->kind.assign(d->kind, d->kind + d->n_pts);
    rc->sid.assign(d->struct_id, d->struct_id + d->n_pts);
    rc->d_presc.assign(d->d_presc, d->d_presc + d->n_targets);
    rc->q_area.assign(d->q_area, d->q_area + d->n_targets);
    rc->q_vol.assign(d->q_vol, d->q_vol + d->n_targets);
    if (d->n_oars) rc->d_oar.assign(d->d_oar, d->d_oar + d->n_oars);
    rc->footprint = request_footprint(d->n_iso, d->n_pts, s.width, s.p.case_params.precision);
    if (rc->footprint > s.budget) {
        set_error("lgk_server_open: case needs ~" + std::to_string(rc->footprint) +
                  " device bytes, more than the server budget of " + std::to_string(s.budget));
        return LGK_EBUDGET;
    }
    {
        std::lock_guard<std::mutex> lk(s.mu);
        rc->id = s.next_id++;
        *case_id = rc->id;
        s.queue.push_back(rc.get());
        s.cases[rc->id] = std::move(rc);
    }
    s.cv_work.notify_all();
    return LGK_OK;
}

int lgk_server_submit_to(lgk_server* h, long long case_id, int K, const double* W, long long* id) {
    if (!h || !W || !id || K < 1 || K > (1 << 20) || !valid_weights(K, W)) {
        set_error("lgk_server_submit_to: invalid argument (1 <= K <= 2^20, weights finite, >= 0, w_BOT > 0)");
        return LGK_EINVAL;
    }
    Server& s = h->s;
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.cases.find(case_id);
    if (it == s.cases.end() || it->second->closed || it->second->finished) {
        set_error("lgk_server_submit_to: unknown or closed case id");
        return LGK_EINVAL;
    }
    if (it->second->status != LGK_OK) {
        set_error("lgk_server_submit_to: the case failed: " + it->second->err);
        return it->second->status;
    }
    s.add_request(*it->second, K, W, id);
    return LGK_OK;
}

int lgk_server_close(lgk_server* h, long long case_id) {
    if (!h) {
        set_error("lgk_server_close: server is NULL");
        return LGK_EINVAL;
    }
    Server& s = h->s;
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.cases.find(case_id);
    if (it == s.cases.end()) {
        set_error("lgk_server_close: unknown case id (or already finished)");
        return LGK_EINVAL;
    }
    it->second->closed = true;
    it->second->cv.notify_all();
    return LGK_OK;
}

int lgk_server_submit(lgk_server* h, const lgk_case_desc* d, int K, const double* W, long long* id) {
    if (!h || !W || !id || K < 1 || K > (1 << 20) || !valid_weights(K, W)) {
        set_error("lgk_server_submit: invalid argument");
        return LGK_EINVAL;
    }
    long long cid = 0;
    int rc = lgk_server_open(h, d, &cid);
    if (rc) return rc;
    Server& s = h->s;
    std::lock_guard<std::mutex> lk(s.mu);
    Resident& r = *s.cases.at(cid);
    s.add_request(r, K, W, id);
    r.closed = true;          // a one-shot request: the case leaves once its weightings are done
    r.cv.notify_all();
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
    if (t) std::copy(q->t.begin(), q->t.end(), t);
    if (tau) std::copy(q->tau.begin(), q->tau.end(), tau);
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
        for (Resident* rc : s.queue) s.fail_case(*rc, LGK_ETIMEOUT, "server destroyed");
        s.queue.clear();
        for (auto& kv : s.cases) kv.second->cv.notify_all();
    }
    s.cv_work.notify_all();
    for (auto& w : s.workers) w.join();
    for (auto& st : s.streams) cudaStreamDestroy(st);
    delete h;
}

}  // extern "C"
