// Two-pass optimisation (Sec. 2.C): low-dose volumes of the first-pass plans
// on the device, non-redundant sampling of their points (Algorithm 1) on the
// host, and the second pass as one masked batched solve over the union of the
// sampled points.
#include <math.h>

#include <algorithm>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "lgk_impl.hpp"

struct lgk_result {
    std::unique_ptr<lgk::ResultData> d;
};

namespace lgk {

// ------------------------------------------------------------ low-dose volumes
// Membership of candidate points in [lo_l, hi_l) for every level l and plan j,
// from the chunk's doses dose[j][e] (e < n_chunk, chunk starting at candidate
// c0, a multiple of 32): one bit per candidate, one warp ballot per word.
// Grid ((n_chunk + 255) / 256, K), 256 threads.
__global__ void k_ld_member(const double* __restrict__ dose, int n_chunk, int c0, int K, int n_lev,
                            const double* __restrict__ lo, const double* __restrict__ hi, int words,
                            uint32_t* member, int* count) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    const double d = e < n_chunk ? dose[(size_t)j * n_chunk + e] : -INFINITY;
    const int w = (c0 + e) >> 5;
    for (int l = 0; l < n_lev; ++l) {
        const bool in = e < n_chunk && d >= lo[l] && d < hi[l];
        const uint32_t bits = __ballot_sync(0xffffffffu, in);
        if ((threadIdx.x & 31) == 0 && e < n_chunk) {
            member[((size_t)l * K + j) * words + w] = bits;
            if (bits) atomicAdd(&count[l * K + j], __popc(bits));
        }
    }
}

int low_dose_volumes(const ResultData& r, const double* phi_cand, int n_cand, int n_lev,
                     const double* d_lo, const double* delta, uint32_t* member, int* count) {
    CaseData& cs = *r.cs;
    cudaStream_t st = cs.stream;
    const int B = cs.n_beams, K = r.K, words = (n_cand + 31) / 32;
    // candidates per chunk: a multiple of 32 with phi and doses under ~256 MiB
    long long per = (256ll << 20) / (8ll * (B + K));
    per = std::max(32ll, per / 32 * 32);
    const int chunk = (int)std::min<long long>(per, round_up(n_cand, 32));
    DevBuf td, pd, dd, lod, hid, mem, cnt;
    int rc;
    if ((rc = td.alloc((size_t)K * B * 8)) || (rc = pd.alloc((size_t)chunk * B * 8)) ||
        (rc = dd.alloc((size_t)K * chunk * 8)) || (rc = lod.alloc((size_t)n_lev * 8)) ||
        (rc = hid.alloc((size_t)n_lev * 8)) || (rc = mem.alloc((size_t)n_lev * K * words * 4)) ||
        (rc = cnt.alloc((size_t)n_lev * K * 4)))
        return rc;
    std::vector<double> hi(n_lev);
    for (int l = 0; l < n_lev; ++l) hi[l] = d_lo[l] + delta[l];
    LGK_CUDA_TRY(cudaMemcpyAsync(lod.p, d_lo, lod.bytes, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(hid.p, hi.data(), hid.bytes, cudaMemcpyHostToDevice, st));
    LGK_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, cnt.bytes, st));
    if ((rc = times_into(r, td.as<double>()))) return rc;
    for (int c0 = 0; c0 < n_cand; c0 += chunk) {
        const int nc = std::min(chunk, n_cand - c0);
        LGK_CUDA_TRY(cudaMemcpyAsync(pd.p, phi_cand + (size_t)c0 * B, (size_t)nc * B * 8,
                                     cudaMemcpyHostToDevice, st));
        // dose[K][nc] = t[K][B] . phi[nc][B]^T (the kernel lgk_fetch_doses uses)
        if ((rc = dgemm(st, false, true, K, nc, B, 1.0, td.as<double>(), B, pd.as<double>(), B, 0.0,
                        dd.as<double>(), nc)))
            return rc;
        dim3 g((nc + 255) / 256, K);
        k_ld_member<<<g, 256, 0, st>>>(dd.as<double>(), nc, c0, K, n_lev, lod.as<double>(),
                                       hid.as<double>(), words, mem.as<uint32_t>(), cnt.as<int>());
        LGK_LAUNCH_CHECK();
        // the host copy of phi must stay valid until the chunk's upload ran
        LGK_CUDA_TRY(cudaStreamSynchronize(st));
    }
    LGK_CUDA_TRY(cudaMemcpyAsync(member, mem.p, mem.bytes, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaMemcpyAsync(count, cnt.p, cnt.bytes, cudaMemcpyDeviceToHost, st));
    LGK_CUDA_TRY(cudaStreamSynchronize(st));
    return LGK_OK;
}

// ------------------------------------------------------------------ sampling
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output of a generator
// whose state is x, i.e. the mix of x + the golden gamma.
static inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Random key of candidate i in draw `s` (0: re-selection from the union's
// points, 1: new points) for volume j of level `level`: a counter-based
// stream, so the draws do not depend on the order the keys are made in.
static inline uint64_t draw_key(uint64_t seed, uint64_t level, uint64_t j, uint64_t s, uint64_t i) {
    return splitmix64(splitmix64(splitmix64(splitmix64(seed) ^ level) ^ (2 * j + s)) ^ i);
}

// round(num / den) with halves rounded up, exactly (num, den >= 0, den > 0).
static inline long long round_ratio(unsigned __int128 num, unsigned __int128 den) {
    return (long long)((2 * num + den) / (2 * den));
}

// The k items of `items` with the smallest keys (ties: smaller index): a
// uniformly random k-subset.
static std::vector<int> pick(const std::vector<int>& items, long long k, uint64_t seed, int level,
                             int j, int s) {
    if (k >= (long long)items.size()) return items;
    std::vector<std::pair<uint64_t, int>> kv(items.size());
    for (size_t q = 0; q < items.size(); ++q)
        kv[q] = {draw_key(seed, (uint64_t)level, (uint64_t)j, (uint64_t)s, (uint64_t)items[q]), items[q]};
    std::nth_element(kv.begin(), kv.begin() + k, kv.end());
    std::vector<int> out(k);
    for (long long q = 0; q < k; ++q) out[q] = kv[q].second;
    return out;
}

// Algorithm 1 over K volumes given as candidate bitsets (member[j][words]).
// Output: the union P of the per-volume samples p_j (ascending candidate
// indices) and, per union point, the bitset of the volumes it was sampled
// for (sel[u][ceil(K/32)]).
int sample_low_dose(int K, int n_cand, const uint32_t* member, const int* n_desired, uint64_t seed,
                    int level, int* n_union, int* union_idx, uint32_t* sel) {
    const int words = (n_cand + 31) / 32, kw = (K + 31) / 32;
    std::vector<long long> vol(K), want(K);
    for (int j = 0; j < K; ++j) {
        long long c = 0;
        for (int w = 0; w < words; ++w) c += __builtin_popcount(member[(size_t)j * words + w]);
        vol[j] = c;
        want[j] = std::min<long long>(std::max(n_desired[j], 0), c);   // omega_j <= 1
    }
    // volumes by decreasing sampling density omega_j = want_j / |V_j| (ties:
    // smaller j); empty volumes have nothing to sample
    std::vector<int> order;
    for (int j = 0; j < K; ++j)
        if (vol[j] > 0) order.push_back(j);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (unsigned __int128)want[a] * vol[b] > (unsigned __int128)want[b] * vol[a];
    });
    auto in_vol = [&](int j, int i) { return (member[(size_t)j * words + (i >> 5)] >> (i & 31)) & 1u; };

    std::vector<uint8_t> in_u(n_cand, 0);          // V^cup
    long long u_size = 0;
    std::vector<int> p_u;                          // p^cup
    std::vector<uint32_t> chosen((size_t)n_cand * kw, 0u);   // candidate x volume: in p_j
    std::vector<uint8_t> in_p(n_cand, 0);          // P
    for (int j : order) {
        // re-selection from the union's points at density omega_j
        long long k1 = round_ratio((unsigned __int128)want[j] * (unsigned long long)u_size,
                                   (unsigned __int128)vol[j]);
        std::vector<int> tilde = pick(p_u, k1, seed, level, j, 0);
        // the new part of V_j
        std::vector<int> fresh;
        for (int w = 0; w < words; ++w) {
            uint32_t bits = member[(size_t)j * words + w];
            while (bits) {
                const int i = w * 32 + __builtin_ctz(bits);
                bits &= bits - 1;
                if (!in_u[i]) fresh.push_back(i);
            }
        }
        long long k2 = round_ratio((unsigned __int128)want[j] * (unsigned long long)fresh.size(),
                                   (unsigned __int128)vol[j]);
        std::vector<int> out = pick(fresh, k2, seed, level, j, 1);
        for (int i : tilde)
            if (in_vol(j, i)) chosen[(size_t)i * kw + (j >> 5)] |= 1u << (j & 31), in_p[i] = 1;
        for (int i : out) chosen[(size_t)i * kw + (j >> 5)] |= 1u << (j & 31), in_p[i] = 1;
        p_u = std::move(tilde);
        p_u.insert(p_u.end(), out.begin(), out.end());
        for (int i : fresh) in_u[i] = 1;
        u_size += (long long)fresh.size();
    }
    int nu = 0;
    for (int i = 0; i < n_cand; ++i) {
        if (!in_p[i]) continue;
        union_idx[nu] = i;
        if (sel) std::copy(&chosen[(size_t)i * kw], &chosen[(size_t)i * kw] + kw, sel + (size_t)nu * kw);
        ++nu;
    }
    *n_union = nu;
    return LGK_OK;
}

}  // namespace lgk

using namespace lgk;

namespace {

int fail2(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

bool all_finite_nonneg(const double* x, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!(x[i] >= 0.0) || !isfinite(x[i])) return false;
    return true;
}

}  // namespace

extern "C" {

int lgk_low_dose_volumes(const lgk_result* res, const double* phi_cand, int n_cand, int n_levels,
                         const double* d_lo, const double* delta, uint32_t* member, int* count) {
    if (!res || !phi_cand || !d_lo || !delta || !member || !count || n_cand < 1 || n_levels < 1 ||
        n_levels > 8)
        return fail2(LGK_EINVAL, "lgk_low_dose_volumes: NULL argument, n_cand < 1 or n_levels not in 1..8");
    for (int l = 0; l < n_levels; ++l)
        if (!(d_lo[l] > 0) || !(delta[l] > 0) || !isfinite(d_lo[l] + delta[l]))
            return fail2(LGK_EINVAL, "lgk_low_dose_volumes: need d_lo > 0 and delta > 0");
    if (int rb = result_ready(*res->d)) return rb;
    const CaseData& cs = *res->d->cs;
    if (!all_finite_nonneg(phi_cand, (size_t)n_cand * cs.n_beams))
        return fail2(LGK_EINVAL, "lgk_low_dose_volumes: phi_cand must be finite and >= 0");
    LGK_CUDA_TRY(cudaSetDevice(cs.device));
    try {
        return low_dose_volumes(*res->d, phi_cand, n_cand, n_levels, d_lo, delta, member, count);
    } catch (const std::bad_alloc&) {
        return fail2(LGK_ENOMEM, "host allocation failed");
    }
}

int lgk_sample_low_dose(int K, int n_cand, const uint32_t* member, const int* n_desired, uint64_t seed,
                        int level, int* n_union, int* union_idx, uint32_t* sel) {
    if (K < 1 || n_cand < 1 || !member || !n_desired || !n_union || !union_idx)
        return fail2(LGK_EINVAL, "lgk_sample_low_dose: NULL argument, K < 1 or n_cand < 1");
    try {
        return sample_low_dose(K, n_cand, member, n_desired, seed, level, n_union, union_idx, sel);
    } catch (const std::bad_alloc&) {
        return fail2(LGK_ENOMEM, "host allocation failed");
    }
}

int lgk_two_pass(const lgk_case_desc* d, const lgk_params* p, int K, const double* W, double w0_bot,
                 double rho0_per_beta, double tol, int max_iter, const lgk_pass2_params* p2,
                 lgk_result** res1_out, lgk_case** case2_out, lgk_result** res2_out, int* n_union,
                 int* union_idx) {
    if (!case2_out || !res2_out) return fail2(LGK_EINVAL, "lgk_two_pass: case2_out / res2_out is NULL");
    *case2_out = nullptr;
    *res2_out = nullptr;
    if (res1_out) *res1_out = nullptr;
    if (!d || !W || !p2 || !p2->phi_cand || p2->n_cand < 1 || !(rho0_per_beta > 0) || !(w0_bot > 0))
        return fail2(LGK_EINVAL, "lgk_two_pass: NULL argument, n_cand < 1, or rho rule constants <= 0");
    if (!(p2->delta_ld1 > 0) || !(p2->delta_ld2 > 0))
        return fail2(LGK_EINVAL, "lgk_two_pass: need delta_ld1 > 0 and delta_ld2 > 0");
    const int P = d->n_pts, B = 24 * d->n_iso, nc = p2->n_cand;
    if (!d->kind || !d->phi) return fail2(LGK_EINVAL, "lgk_two_pass: case description incomplete");
    int rc;
    // pass 1: the points as given (low-dose points from a geometric expansion)
    lgk_case* c1 = nullptr;
    lgk_result* r1 = nullptr;
    std::unique_ptr<lgk_case, void (*)(lgk_case*)> c1_guard(nullptr, lgk_destroy_case);
    std::unique_ptr<lgk_result, void (*)(lgk_result*)> r1_guard(nullptr, lgk_free_result);
    if ((rc = lgk_create_case(d, p, &c1))) return rc;
    c1_guard.reset(c1);
    double beta1 = 1.0;
    lgk_case_info(c1, nullptr, nullptr, &beta1, nullptr);
    if ((rc = lgk_solve_weightings(c1, K, W, nullptr, w0_bot, rho0_per_beta * beta1, tol, max_iter, &r1)))
        return rc;
    r1_guard.reset(r1);
    // low-dose volumes [D_LD, D_LD + Delta) of every first-pass plan
    const int words = (nc + 31) / 32, kw = (K + 31) / 32;
    std::vector<uint32_t> member((size_t)2 * K * words);
    std::vector<int> vcount((size_t)2 * K);
    const double lo[2] = {d->d_ld1, d->d_ld2}, dl[2] = {p2->delta_ld1, p2->delta_ld2};
    if ((rc = lgk_low_dose_volumes(r1, p2->phi_cand, nc, 2, lo, dl, member.data(), vcount.data())))
        return rc;
    // Algorithm 1 per level; desired counts default to the first pass's
    int n1[2] = {0, 0};
    for (int q = 0; q < P; ++q) n1[0] += d->kind[q] == LGK_LD1, n1[1] += d->kind[q] == LGK_LD2;
    std::vector<int> uidx((size_t)2 * nc), nu(2);
    std::vector<uint32_t> sel((size_t)2 * nc * kw);
    for (int l = 0; l < 2; ++l) {
        const int want = (l == 0 ? p2->n_ld1 : p2->n_ld2) > 0 ? (l == 0 ? p2->n_ld1 : p2->n_ld2) : n1[l];
        std::vector<int> nd(K, want);
        if ((rc = lgk_sample_low_dose(K, nc, member.data() + (size_t)l * K * words, nd.data(), p2->seed, l,
                                      &nu[l], uidx.data() + (size_t)l * nc, sel.data() + (size_t)l * nc * kw)))
            return rc;
    }
    // pass-2 points: the first pass's non-low-dose points, then the LD1 and
    // LD2 union points; mask rows: all weightings for the kept points, the
    // sampled weightings for the union points
    std::vector<int> keep;
    for (int q = 0; q < P; ++q)
        if (d->kind[q] != LGK_LD1 && d->kind[q] != LGK_LD2) keep.push_back(q);
    const int P2 = (int)keep.size() + nu[0] + nu[1];
    std::vector<double> phi2((size_t)P2 * B);
    std::vector<uint8_t> kind2(P2);
    std::vector<uint16_t> sid2(P2, 0);
    std::vector<uint32_t> mask2((size_t)P2 * kw, 0u);
    int q2 = 0;
    for (int q : keep) {
        std::copy(d->phi + (size_t)q * B, d->phi + (size_t)(q + 1) * B, &phi2[(size_t)q2 * B]);
        kind2[q2] = d->kind[q];
        sid2[q2] = d->struct_id ? d->struct_id[q] : 0;
        for (int w = 0; w < kw; ++w) mask2[(size_t)q2 * kw + w] = 0xffffffffu;
        ++q2;
    }
    for (int l = 0; l < 2; ++l)
        for (int u = 0; u < nu[l]; ++u) {
            const int i = uidx[(size_t)l * nc + u];
            std::copy(p2->phi_cand + (size_t)i * B, p2->phi_cand + (size_t)(i + 1) * B, &phi2[(size_t)q2 * B]);
            kind2[q2] = l == 0 ? LGK_LD1 : LGK_LD2;
            std::copy(&sel[((size_t)l * nc + u) * kw], &sel[((size_t)l * nc + u) * kw] + kw,
                      &mask2[(size_t)q2 * kw]);
            ++q2;
        }
    lgk_case_desc d2 = *d;
    d2.n_pts = P2;
    d2.phi = phi2.data();
    d2.kind = kind2.data();
    d2.struct_id = sid2.data();
    lgk_case* c2 = nullptr;
    lgk_result* r2 = nullptr;
    if ((rc = lgk_create_case(&d2, p, &c2))) return rc;
    double beta2 = 1.0;
    lgk_case_info(c2, nullptr, nullptr, &beta2, nullptr);
    if ((rc = lgk_solve_weightings_masked(c2, K, W, nullptr, w0_bot, rho0_per_beta * beta2, tol, max_iter,
                                          mask2.data(), nullptr, nullptr, &r2))) {
        lgk_destroy_case(c2);
        return rc;
    }
    if (n_union) n_union[0] = nu[0], n_union[1] = nu[1];
    if (union_idx)
        for (int l = 0; l < 2; ++l)
            std::copy(&uidx[(size_t)l * nc], &uidx[(size_t)l * nc] + nu[l], union_idx + (size_t)l * nc);
    if (res1_out) *res1_out = r1_guard.release();
    *case2_out = c2;
    *res2_out = r2;
    return LGK_OK;
}

}  // extern "C"
