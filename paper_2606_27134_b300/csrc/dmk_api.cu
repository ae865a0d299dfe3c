// C ABI of the periodized DMK library: plan construction, workspace, and the evaluation
// sequence (tree -> upward -> root -> plane waves -> shift -> leaf) on the plan's stream.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_select.cuh>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <mutex>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "dmk_internal.h"
#include "dmk_fast.cuh"

using namespace dmk;

namespace {

thread_local std::string g_plan_error;

// Static device workspace of dmk_eval_static (see include/dmk.h): every GPU that loads the
// library holds these bytes until the process exits.  Host code only ever sees the address
// returned by cudaGetSymbolAddress for the current device.
constexpr size_t kStaticWorkspaceBytes = (size_t)64 << 20;
constexpr int64_t kStaticMaxN = 16384;
static __device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];
constexpr int kMaxDevices = 64;
void* g_static_ptr[kMaxDevices] = {};
std::mutex g_static_mu;

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

}  // namespace

struct dmk_plan_s {
    PlanTables T;
    int prec = DMK_MIXED;
    int n_s = 250;
    cudaStream_t stream = nullptr;
    Geo geo{};
    std::string err;
    dmk_stats_t stats{};
    int timing = 0;
    int device = 0;
    size_t smem_optin = 0;
    // device tables
    void* d_tab64 = nullptr;
    void* d_tab32 = nullptr;
    Tab<double> tab64{};
    Tab<float> tab32{};
    void* d_root = nullptr;
    RootTab root{};
    RootTab root2{};                // second root part (original symbol), nmode = 0 if none
    void* d_root2 = nullptr;
    double* d_self = nullptr;      // self_val then self_grad
    int* d_cube = nullptr;         // non-exact tilings: cube classes (Mtot), then the cut-cube count and list
    // workspace
    std::vector<DevBuf> bufs;
    unsigned char* h_meta = nullptr;   // pinned host staging for the small per-evaluation readbacks
    double* h_chi = nullptr;           // pinned host staging of a shard's structure factor
    size_t h_chi_cap = 0;
    cudaEvent_t ev[11] = {};
    // residual sums (k_pair) run on their own stream beside the far field when pair_overlap is
    // set, at most pair_blocks resident blocks per SM (0: as many as fit).  On by default with
    // no cap: the far-field kernels of the direct path leave room on the SMs (measured: headline
    // slab -8 %, clustered -3 %, Stokeslet 1P -2 %, rotlet 16 cubes -1 % per evaluation); the
    // results are the same bits either way (k_pair stores, the expansions add after the join)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_cnt = nullptr;
    int pair_overlap = 1;
    int pair_blocks = 0;
    int n_sm = 148;                 // replaced by the device's SM count at plan creation
    // resident blocks per SM of the persistent kernels, by kernel
    std::unordered_map<const void*, int> occ;
    int launches = 0;
    // device allocations made by this plan so far (cudaMalloc, cudaMallocAsync)
    int64_t n_allocs = 0;
    // set by dmk_vjp while it evaluates with the upstream gradient as strengths: the net
    // charge of Laplace D = 1, 2 is then allowed (only gradients of the result are used)
    int allow_charged = 0;
    // set only while dmk_eval_static runs: device buffers are carved from this range
    unsigned char* arena = nullptr;
    size_t arena_cap = 0, arena_off = 0;
    // dynamic shared memory already opted in per kernel (the attribute persists on the device)
    std::unordered_map<const void*, size_t> smem_set;

};

namespace {

#define CK(call)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            plan->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
            return e_ == cudaErrorMemoryAllocation ? DMK_ERR_OOM : DMK_ERR_CUDA;  \
        }                                                                         \
    } while (0)

#define CKS(x)                              \
    do {                                    \
        dmk_status_t s_ = (x);              \
        if (s_ != DMK_OK) return s_;        \
    } while (0)

enum BufId {
    B_W, B_KEYS, B_KEYS2, B_IDX, B_IDX2, B_XS, B_RS, B_CUB, B_FLAGS, B_CNT,
    B_CELLS, B_R, B_CAND, B_BOXU64, B_BOXINT, B_LEAVES, B_DOFFS, B_DL, B_NLBOX, B_TASKS, B_BAL,
    B_PROXY, B_LOCAL, B_PW, B_SCRATCH, B_CHI, B_UHAT, B_MISC, B_DEVPTS, B_DEVRHO, B_DEVPOT, B_DEVGRAD, B_XF, B_VW, B_PART,
    B_VJPV, B_VJPG, B_VJPQ, B_ICNT, B_SRC, B_ORIG, B_CHIP, B_SHARDCLS, B_TPTS, B_TRHO, B_ITEMS,
    B_COUNT
};

// carve `bytes` (rounded to 256) from the static workspace of dmk_eval_static
dmk_status_t arena_take(dmk_plan_s* plan, size_t bytes, void** out) {
    size_t need = (std::max<size_t>(bytes, 16) + 255) & ~(size_t)255;
    if (plan->arena_off + need > plan->arena_cap) {
        plan->err = "dmk_eval_static: this problem needs more than the " + std::to_string(plan->arena_cap >> 20) +
                    " MiB static workspace";
        return DMK_ERR_OOM;
    }
    *out = plan->arena + plan->arena_off;
    plan->arena_off += need;
    return DMK_OK;
}

// Waits for the small readback just queued on st.  These complete within tens of
// microseconds, and a blocking wait was measured to return up to ~70 us after the copy had
// finished, so the host polls first (at most 2 ms) and only then blocks.
dmk_status_t host_wait(dmk_plan_s* plan, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        const cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) return DMK_OK;
        if (e != cudaErrorNotReady) CK(e);
        if (std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(2000)) break;
    }
    CK(cudaStreamSynchronize(st));
    return DMK_OK;
}

// the same for an event
dmk_status_t host_wait_event(dmk_plan_s* plan, cudaEvent_t ev) {
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return DMK_OK;
        if (e != cudaErrorNotReady) CK(e);
        if (std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(2000)) break;
    }
    CK(cudaEventSynchronize(ev));
    return DMK_OK;
}

dmk_status_t ensure(dmk_plan_s* plan, int id, size_t bytes, void** out) {
    if (plan->bufs.size() < B_COUNT) plan->bufs.resize(B_COUNT);
    DevBuf& b = plan->bufs[id];
    if (bytes == 0) bytes = 16;
    if (plan->arena) {
        if (b.cap < bytes) {
            dmk_status_t s = arena_take(plan, bytes, &b.p);
            if (s != DMK_OK) return s;
            b.cap = (bytes + 255) & ~(size_t)255;
        }
        *out = b.p;
        return DMK_OK;
    }
    if (b.cap < bytes) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
        size_t want = bytes + bytes / 4;
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            plan->err = "device allocation of " + std::to_string(want) + " bytes failed";
            return DMK_ERR_OOM;
        }
        ++plan->n_allocs;
        b.cap = want;
    }
    *out = b.p;
    return DMK_OK;
}

// value and t-derivative of sum_n a_n T_n(t) (T_n' = n U_{n-1})
void cheb_value_deriv(const std::vector<double>& a, double t, double& v, double& d) {
    double tm1 = 1, tm2 = 0, um1 = 1, um2 = 0;   // T_{n-1}, T_{n-2}, U_{n-1}, U_{n-2}
    v = 0;
    d = 0;
    for (size_t n = 0; n < a.size(); ++n) {
        double tn, un;
        if (n == 0) { tn = 1; un = 1; }
        else if (n == 1) { tn = t; un = 2 * t; tm2 = 1; um2 = 1; }
        else { tn = 2 * t * tm1 - tm2; un = 2 * t * um1 - um2; tm2 = tm1; um2 = um1; }
        v += a[n] * tn;
        if (n > 0) d += a[n] * (double)n * (n == 1 ? 1.0 : um1);
        tm1 = tn;
        um1 = un;
    }
}

// Piecewise cubic Hermite tables of the six residual series q, f, g, q', f', g' on s in [0, 1]
// (App. B residual functions as precomputed polynomial approximations): kHermNT intervals, the
// interval i holding (c0, c1, c2, c3) with X = c0 + u (c1 + u (c2 + u c3)), u = s kHermNT - i,
// matching the FP64 series value and s-derivative at both interval ends.
std::vector<double> herm_tables(const PlanTables& P) {
    const std::vector<double>* ser[6] = {&P.fit_q, &P.fit_f, &P.fit_g, &P.fit_dq, &P.fit_df, &P.fit_dg};
    std::vector<double> out((size_t)6 * kHermNT * 4, 0.0);
    std::vector<double> v(kHermNT + 1), d(kHermNT + 1);
    for (int k = 0; k < 6; ++k) {
        if (ser[k]->empty()) continue;
        for (int j = 0; j <= kHermNT; ++j) {
            const double sj = (double)j / kHermNT;
            cheb_value_deriv(*ser[k], 2 * sj - 1, v[j], d[j]);
            d[j] *= 2.0 / kHermNT;      // d/du = (d/ds) / kHermNT, d/ds = 2 d/dt
        }
        for (int i = 0; i < kHermNT; ++i) {
            double* c = &out[((size_t)k * kHermNT + i) * 4];
            c[0] = v[i];
            c[1] = d[i];
            c[2] = 3 * (v[i + 1] - v[i]) - 2 * d[i] - d[i + 1];
            c[3] = 2 * (v[i] - v[i + 1]) + d[i] + d[i + 1];
        }
    }
    return out;
}

template <class T>
dmk_status_t upload_tab(dmk_plan_s* plan, void** mem, Tab<T>& tab, double fit_tol) {
    const PlanTables& P = plan->T;
    const int p = P.p;
    auto trunc = [&](const std::vector<double>& a) {
        double mx = 0;
        for (double v : a) mx = std::max(mx, std::fabs(v));
        int n = (int)a.size();
        while (n > 1 && std::fabs(a[n - 1]) < fit_tol * mx) --n;
        return std::vector<double>(a.begin(), a.begin() + n);
    };
    std::vector<std::vector<double>> fits = {trunc(P.fit_q), trunc(P.fit_f), trunc(P.fit_g),
                                             trunc(P.fit_dq), trunc(P.fit_df), trunc(P.fit_dg)};
    size_t nfit = 0;
    for (auto& f : fits) nfit += f.size();
    if (nfit > 256) { plan->err = "residual fits longer than 256 coefficients"; return DMK_ERR_INVALID_ARG; }
    std::vector<T> h;
    auto push = [&](const std::vector<double>& v) {
        size_t o = h.size();
        for (double x : v) h.push_back((T)x);
        while (h.size() % 4) h.push_back(0);
        return o;
    };
    size_t o_nodes = push(P.nodes), o_bary = push(P.bary), o_I = push(P.Ioct), o_C = push(P.Cm);
    size_t o_A = push(P.Aoct);
    std::vector<double> Eri;
    for (auto& z : P.E) { Eri.push_back(z.real()); Eri.push_back(z.imag()); }
    size_t o_E = push(Eri), o_g = push(P.gdiff);
    size_t o_fit = h.size();
    int offs[6], lens[6];
    size_t acc = 0;
    for (int i = 0; i < 6; ++i) {
        offs[i] = (int)acc;
        lens[i] = (int)fits[i].size();
        for (double x : fits[i]) h.push_back((T)x);
        acc += fits[i].size();
    }
    while (h.size() % 4) h.push_back(0);
    // FP32 path: cubic tables, 16-byte aligned
    size_t o_herm = h.size();
    if (sizeof(T) == 4) {
        std::vector<double> ht = herm_tables(P);
        for (double x : ht) h.push_back((T)x);
    }
    cudaError_t e = cudaMalloc(mem, h.size() * sizeof(T));
    if (e != cudaSuccess) { plan->err = "table allocation failed"; return DMK_ERR_OOM; }
    ++plan->n_allocs;
    e = cudaMemcpy(*mem, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { plan->err = cudaGetErrorString(e); return DMK_ERR_CUDA; }
    T* base = (T*)*mem;
    tab.p = p; tab.nf = P.nf; tab.NF = P.NF; tab.nfh = P.nfh;
    tab.d_rho = P.d_rho; tab.d_u = P.d_u; tab.kernel = P.kernel; tab.level_power = P.level_power;
    tab.nodes = base + o_nodes; tab.bary = base + o_bary; tab.Ioct = base + o_I; tab.Cm = base + o_C;
    tab.Aoct = base + o_A;
    tab.E = reinterpret_cast<const Cx<T>*>(base + o_E);
    tab.gdiff = base + o_g;
    tab.fit = base + o_fit;
    tab.herm = (sizeof(T) == 4) ? reinterpret_cast<const float*>(base + o_herm) : nullptr;
    tab.off_q = offs[0]; tab.n_q = lens[0]; tab.off_f = offs[1]; tab.n_f = lens[1];
    tab.off_g = offs[2]; tab.n_g = lens[2]; tab.off_dq = offs[3]; tab.n_dq = lens[3];
    tab.off_df = offs[4]; tab.n_df = lens[4]; tab.off_dg = offs[5]; tab.n_dg = lens[5];
    return DMK_OK;
}

// one root part (wavenumber axes, weights on their rectangle, cube-index DFT lengths Q or
// nullptr) as a device table
dmk_status_t upload_root_part(dmk_plan_s* plan, const std::vector<double>* kax, const std::vector<std::complex<double>>& Wr,
                              const int* Q, void** dptr, RootTab& rt) {
    const PlanTables& P = plan->T;
    const int p = P.p;
    std::vector<double> h;
    auto pad = [&]() { while (h.size() % 2) h.push_back(0); };
    size_t o_k[3], o_S[3];
    for (int i = 0; i < 3; ++i) {
        o_k[i] = h.size();
        for (double v : kax[i]) h.push_back(v);
        pad();
    }
    for (int i = 0; i < 3; ++i) {
        o_S[i] = h.size();
        for (double k : kax[i])
            for (int j = 0; j < p; ++j) {
                double ph = -k * (P.s / 2) * P.nodes[j];
                h.push_back(std::cos(ph));
                h.push_back(std::sin(ph));
            }
    }
    size_t o_W = h.size();
    for (auto& z : Wr) { h.push_back(z.real()); h.push_back(z.imag()); }
    size_t o_c = h.size();
    for (double v : P.root_const) h.push_back(v);
    // per axis: exp(2 pi i t / Q), t = 0..Q-1, and n mod Q for every wavenumber k = 2 pi n / (Q s)
    size_t o_r[3], o_n[3];
    int Qa[3];
    for (int a = 0; a < 3; ++a) {
        Qa[a] = Q && Q[a] > 0 ? Q[a] : 1;
        pad();
        o_r[a] = h.size();
        for (int t = 0; t < Qa[a]; ++t) {
            const double ang = 2 * 3.14159265358979323846 * (double)t / Qa[a];
            h.push_back(std::cos(ang));
            h.push_back(std::sin(ang));
        }
        o_n[a] = h.size();
        for (double k : kax[a]) {
            const long long n = std::llround(k * Qa[a] * P.s / (2 * 3.14159265358979323846));
            h.push_back((double)(((n % Qa[a]) + Qa[a]) % Qa[a]));
        }
    }
    cudaError_t e = cudaMalloc(dptr, h.size() * sizeof(double));
    if (e != cudaSuccess) { plan->err = "root table allocation failed"; return DMK_ERR_OOM; }
    ++plan->n_allocs;
    e = cudaMemcpy(*dptr, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { plan->err = cudaGetErrorString(e); return DMK_ERR_CUDA; }
    double* base = (double*)*dptr;
    rt.n1 = (int)kax[0].size(); rt.n2 = (int)kax[1].size(); rt.n3 = (int)kax[2].size();
    rt.nmode = rt.n1 * rt.n2 * rt.n3;
    for (int i = 0; i < 3; ++i) {
        rt.kax[i] = base + o_k[i];
        rt.S[i] = reinterpret_cast<const Cx<double>*>(base + o_S[i]);
    }
    rt.W = reinterpret_cast<const Cx<double>*>(base + o_W);
    rt.rconst = base + o_c;
    for (int a = 0; a < 3; ++a) {
        rt.Q[a] = Qa[a];
        rt.nmod[a] = base + o_n[a];
        rt.roots[a] = reinterpret_cast<const Cx<double>*>(base + o_r[a]);
    }
    return DMK_OK;
}

dmk_status_t upload_root(dmk_plan_s* plan) {
    const PlanTables& P = plan->T;
    CKS(upload_root_part(plan, P.kax, P.Wroot, P.root_dft ? P.root_dft_Q[0] : nullptr, &plan->d_root, plan->root));
    plan->root2 = RootTab{};
    if (P.original_symbol)
        CKS(upload_root_part(plan, P.kax2, P.Wroot2, P.root_dft ? P.root_dft_Q[1] : nullptr, &plan->d_root2,
                             plan->root2));
    cudaError_t e;
    // self tables
    std::vector<double> sv(P.self_val);
    sv.insert(sv.end(), P.self_grad.begin(), P.self_grad.end());
    e = cudaMalloc(&plan->d_self, sv.size() * sizeof(double));
    if (e != cudaSuccess) { plan->err = "self table allocation failed"; return DMK_ERR_OOM; }
    ++plan->n_allocs;
    cudaMemcpy(plan->d_self, sv.data(), sv.size() * sizeof(double), cudaMemcpyHostToDevice);
    return DMK_OK;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// work-buffer placement: dynamic shared memory when it fits, else a global scratch slice
struct Place {
    int use_smem;
    size_t bytes;
    unsigned grid;
};

template <class T>
struct Evaluator {
    dmk_plan_s* plan;
    Tab<T>& tab;
    Evaluator(dmk_plan_s* pl, Tab<T>& t) : plan(pl), tab(t) {}

    dmk_status_t place(size_t bytes, int n, Place& pl, unsigned char** scratch) {
        // kernels using place() have at most a few hundred bytes of static shared memory
        const size_t lim = plan->smem_optin > 4096 ? plan->smem_optin - 4096 : 0;
        pl.bytes = bytes;
        pl.grid = (unsigned)std::max(1, std::min<int>(n, plan->n_sm * 8));
        if (bytes <= lim) {
            pl.use_smem = 1;
            *scratch = nullptr;
            return DMK_OK;
        }
        pl.use_smem = 0;
        // the static workspace of dmk_eval_static holds at most 16 per-CTA slices
        pl.grid = (unsigned)std::max(1, std::min<int>(n, plan->arena ? 16 : plan->n_sm * 2));
        void* p = nullptr;
        dmk_status_t s = ensure(plan, B_SCRATCH, bytes * pl.grid, &p);
        *scratch = (unsigned char*)p;
        return s;
    }
};

// opt in to `bytes` of dynamic shared memory (without it the limit is 48 KB minus the static part)
template <class K>
dmk_status_t set_smem(dmk_plan_s* plan, K kernel, size_t bytes) {
    if (bytes == 0) return DMK_OK;
    size_t& done = plan->smem_set[(const void*)kernel];
    if (bytes <= done) return DMK_OK;
    CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done = bytes;
    return DMK_OK;
}

template <class T, int MAXP>
dmk_status_t launch_anterp(dmk_plan_s* plan, Tab<T>& tab, int nleaf_cap, const int* nleaf_dev, const int* leaves,
                           BoxArrays B, const double* xs, int64_t N, const double* rs, T* proxy) {
    const int p2 = tab.p * tab.p;
    int threads = std::min(MAXP <= 24 ? 576 : 512, ((p2 + 31) / 32) * 32);
    size_t sm = 3 * (size_t)kAnterpChunk * MAXP * sizeof(T);
    CKS(set_smem(plan, k_anterp<T, MAXP>, sm));
    unsigned grid = (unsigned)std::max(1, std::min(nleaf_cap, plan->n_sm * 8));
    k_anterp<T, MAXP><<<grid, threads, sm, plan->stream>>>(nleaf_dev, leaves, B, xs, N, rs, tab, plan->T.s, proxy,
                                                           nullptr, 0);
    return DMK_OK;
}

template <class T, int MAXP>
dmk_status_t launch_anterp2(dmk_plan_s* plan, Tab<T>& tab, int nleaf_cap, const int* nleaf_dev, const int* leaves,
                            BoxArrays B, const double* xs, int64_t N, const double* rs, T* proxy) {
    const int threads = (((tab.p + 1) / 2) * tab.p + 31) / 32 * 32;
    const size_t sm = 3 * (size_t)kAnterpChunk * MAXP * sizeof(T);
    CKS(set_smem(plan, k_anterp2<T, MAXP>, sm));
    const unsigned grid = (unsigned)std::max(1, std::min(nleaf_cap, plan->n_sm * 8));
    k_anterp2<T, MAXP><<<grid, threads, sm, plan->stream>>>(nleaf_dev, leaves, B, xs, N, rs, tab, plan->T.s, proxy);
    return DMK_OK;
}

// resident blocks per SM of a kernel at a block size and dynamic shared memory (cached per plan)
template <class Kern>
dmk_status_t resident_blocks(dmk_plan_s* plan, Kern kernel, int threads, size_t smem, int* out) {
    auto it = plan->occ.find((const void*)kernel);
    if (it != plan->occ.end()) { *out = it->second; return DMK_OK; }
    int n = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem));
    plan->occ[(const void*)kernel] = *out = std::max(1, n);
    return DMK_OK;
}

// residual sums (k_pair, persistent: every resident block takes tasks from the counter) on
// stream sp
template <class T, int K, bool G>
dmk_status_t launch_pair(dmk_plan_s* plan, Tab<T>& tab, const int* leaves, BoxArrays B, const double* xs, int64_t N,
                         const int* doffs, const DirectEntry* dl, LeafOut lo, const int* toffs, int tcap,
                         const int4* tasks, int* next, cudaStream_t sp) {
    constexpr int DR = Pair<T, K, G>::DR;
    const size_t sm = pair_smem<T, DR>();
    CKS(set_smem(plan, k_pair<T, K, G>, sm));
    int per_sm = 1;
    CKS(resident_blocks(plan, k_pair<T, K, G>, kPairWarps * 32, sm, &per_sm));
    if (plan->pair_overlap && plan->pair_blocks > 0) per_sm = std::min(per_sm, plan->pair_blocks);
    k_pair<T, K, G><<<per_sm * plan->n_sm, kPairWarps * 32, sm, sp>>>(leaves, B, tab, plan->geo, xs, N, doffs, toffs,
                                                                      tcap, tasks, next, dl, lo);
    return DMK_OK;
}

// leaf expansions + residual sums + self terms (k_leafexp)
template <class T, int K, bool G>
dmk_status_t launch_leafexp(dmk_plan_s* plan, Tab<T>& tab, int nleaf, const int* leaves, BoxArrays B, const T* local,
                            const double* xs, int64_t N, LeafOut lo, int direct_leaf, int n_nl, const int* nl_box,
                            int n_root, const int* woff) {
    const size_t se = leafexp_smem<T>(tab.p);
    if (direct_leaf) {
        // chunks of targets of the non-leaf boxes with leaf children and of the cubes that are
        // leaves; at most N / kLeafExpThreads + n_nl + n_root of them
        CKS(set_smem(plan, k_leafexp_parent<T, K, G>, se));
        const int64_t most = N / kLeafExpThreads + n_nl + n_root;
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(most, (int64_t)plan->n_sm * 16));
        k_leafexp_parent<T, K, G><<<grid, kLeafExpThreads, se, plan->stream>>>(n_nl, nl_box, n_root, woff, B, tab,
                                                                               plan->geo, local, xs, N, lo);
        return DMK_OK;
    }
    CKS(set_smem(plan, k_leafexp<T, K, G>, se));
    const unsigned grid = (unsigned)std::max(1, std::min(nleaf, plan->n_sm * 16));
    k_leafexp<T, K, G><<<grid, kLeafExpThreads, se, plan->stream>>>(nleaf, leaves, B, tab, plan->geo, local, xs, N, lo,
                                                                    0);
    return DMK_OK;
}

template <class T, int K>
dmk_status_t launch_leaf(dmk_plan_s* plan, Tab<T>& tab, int nleaf, const int* leaves, BoxArrays B, const T* local,
                         const double* xs, int64_t N, const int* doffs, const DirectEntry* dl, LeafOut lo, bool grad) {
    constexpr int DR = (K == DMK_LAPLACE) ? 1 : (K == DMK_STRESSLET ? 9 : 3);
    const unsigned grid = (unsigned)std::max(1, std::min(nleaf, plan->n_sm * 16));
    const size_t dyn = (size_t)kSrcChunk * kLeaf2Threads + (size_t)kSrcChunk * DR * sizeof(T);
    if (grad) {
        CKS(set_smem(plan, k_leaf2<T, K, true>, dyn));
        k_leaf2<T, K, true><<<grid, kLeaf2Threads, dyn, plan->stream>>>(nleaf, leaves, B, tab, plan->geo, local, xs, N,
                                                                        doffs, dl, lo);
    } else {
        CKS(set_smem(plan, k_leaf2<T, K, false>, dyn));
        k_leaf2<T, K, false><<<grid, kLeaf2Threads, dyn, plan->stream>>>(nleaf, leaves, B, tab, plan->geo, local, xs,
                                                                         N, doffs, dl, lo);
    }
    return DMK_OK;
}

struct TreeInfo {
    int nlev = 0;                 // number of levels
    std::vector<int> ncell, off, nR, nl_off;
    int nb = 0, n_nl = 0, n_leafp = 0;
    int64_t n_entries = 0;
    unsigned long long n_pairs = 0;
};


// Variants of one evaluation (nullptr: every point a target, every cube counted):
//   separate targets (dmk_eval_targets): the targets are the first n_out points, with zero
//       strengths; outputs for them only;
//   one rank of a cube-sharded evaluation (dmk_eval_shard): outputs for the first n_out points
//       (the owned ones), strength sums over them, structure factor over the owned cubes,
//       completed by the caller's reduction.
struct EvalOpts {
    int64_t n_out;              // points with outputs: input index < n_out
    int64_t n_sum;              // strength sums over input index < n_sum
    const int* cube_owned;      // host, Mtot flags, or nullptr (every cube)
    dmk_chi_reduce_fn reduce;   // or nullptr (no reduction)
    void* ctx;
};

// a shard's partial structure factor (n doubles at chi, device) and its strength sums (2 d_rho
// doubles at sums, device) summed over the ranks by the caller's reduction; nothing without one
dmk_status_t reduce_chi(dmk_plan_s* plan, const EvalOpts* sh, Cx<double>* chi, int64_t n, double* sums) {
    if (!sh || !sh->reduce) return DMK_OK;
    const int ns = 2 * plan->T.d_rho;
    const int64_t ntot = n + ns;
    // through plan-owned pinned host memory, so that any host-side all-reduce can serve
    if (plan->h_chi_cap < (size_t)ntot) {
        if (plan->h_chi) cudaFreeHost(plan->h_chi);
        plan->h_chi = nullptr;
        plan->h_chi_cap = 0;
        if (cudaMallocHost((void**)&plan->h_chi, (size_t)ntot * sizeof(double)) != cudaSuccess) {
            plan->h_chi = nullptr;
            plan->err = "pinned host allocation for the structure factor failed";
            return DMK_ERR_OOM;
        }
        plan->h_chi_cap = (size_t)ntot;
    }
    CK(cudaMemcpyAsync(plan->h_chi, chi, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, plan->stream));
    CK(cudaMemcpyAsync(plan->h_chi + n, sums, (size_t)ns * sizeof(double), cudaMemcpyDeviceToHost, plan->stream));
    CK(cudaStreamSynchronize(plan->stream));
    if (sh->reduce(plan->h_chi, ntot, sh->ctx) != 0) {
        plan->err = "the structure-factor reduction of dmk_eval_shard failed";
        return DMK_ERR_CUDA;
    }
    CK(cudaMemcpyAsync(chi, plan->h_chi, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, plan->stream));
    CK(cudaMemcpyAsync(sums, plan->h_chi + n, (size_t)ns * sizeof(double), cudaMemcpyHostToDevice, plan->stream));
    return DMK_OK;
}

template <class T>
dmk_status_t run_eval(dmk_plan_s* plan, Tab<T>& tab, int64_t N0, const double* pts, const double* rho, double* pot,
                      double* grad, const EvalOpts* sh = nullptr) {
    cudaStream_t st = plan->stream;
    const PlanTables& P = plan->T;
    const int drho = P.d_rho, du = P.d_u, p = P.p, p3 = p * p * p;
    const Geo g = plan->geo;
    const int Mtot = g.M[0] * g.M[1] * g.M[2];
    const bool padded = g.padded[0] || g.padded[1] || g.padded[2];
    int launches = 0;
    auto rec = [&](int i) { if (plan->timing) cudaEventRecord(plan->ev[i], st); };
    rec(0);
    // ---- (0) non-exact tilings: the periodic images of the sources in Omega_ext (Sec. 4.1.2)
    // are appended to the N0 points as extra sources; N counts both
    int64_t N = N0;
    void *vmisc, *vsrc = nullptr, *vicnt = nullptr;
    CKS(ensure(plan, B_MISC, 4096, &vmisc));
    // the previous evaluation's residual kernel (side stream) is done with the workspace
    CK(cudaStreamWaitEvent(st, plan->ev_join, 0));
    CK(cudaMemsetAsync(vmisc, 0, 2048, st));
    if (padded) {
        CKS(ensure(plan, B_ICNT, (size_t)(N0 + 1) * 2 * sizeof(int), &vicnt));
        int* icnt = (int*)vicnt;
        int* ioff = icnt + N0 + 1;
        CK(cudaMemsetAsync(icnt + N0, 0, sizeof(int), st));
        k_images<false><<<nblk(N0, 256), 256, 0, st>>>(N0, pts, g, nullptr, 0, icnt, nullptr, nullptr, nullptr,
                                                        nullptr);
        size_t tb = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, tb, icnt, ioff, (int)(N0 + 1), st);
        void* vtmp;
        CKS(ensure(plan, B_CUB, std::max<size_t>(tb, 1 << 20), &vtmp));
        CK(cub::DeviceScan::ExclusiveSum(vtmp, tb, icnt, ioff, (int)(N0 + 1), st));
        CK(cudaMemcpyAsync(plan->h_meta, ioff + N0, sizeof(int), cudaMemcpyDeviceToHost, st));
        CKS(host_wait(plan, st));
        int nimg = 0;
        std::memcpy(&nimg, plan->h_meta, sizeof(int));
        N = N0 + nimg;
        if (N > ((int64_t)1 << 30)) { plan->err = "more than 2^30 points with the periodic images"; return DMK_ERR_INVALID_ARG; }
        launches += 3;
    }
    // ---- (1) keys, sort, gather --------------------------------------------------------
    void *vw, *vkeys, *vkeys2, *vidx, *vidx2, *vxs, *vrs;
    CKS(ensure(plan, B_W, 3 * N * sizeof(double), &vw));
    CKS(ensure(plan, B_KEYS, N * sizeof(uint64_t), &vkeys));
    CKS(ensure(plan, B_KEYS2, N * sizeof(uint64_t), &vkeys2));
    CKS(ensure(plan, B_IDX, N * sizeof(int), &vidx));
    CKS(ensure(plan, B_IDX2, N * sizeof(int), &vidx2));
    CKS(ensure(plan, B_XS, 3 * N * sizeof(double), &vxs));
    CKS(ensure(plan, B_RS, N * drho * sizeof(double), &vrs));
    int* d_err = (int*)vmisc;
    double* d_sums = (double*)((char*)vmisc + 256);          // 2*drho doubles
    unsigned long long* d_pairs = (unsigned long long*)((char*)vmisc + 768);
    uint64_t* keys = (uint64_t*)vkeys;
    uint64_t* keys2 = (uint64_t*)vkeys2;
    int* idx = (int*)vidx;
    int* idx2 = (int*)vidx2;
    double* xs = (double*)vxs;
    double* rs = (double*)vrs;
    k_quantize<<<nblk(N0, 256), 256, 0, st>>>(N0, pts, g, (double*)vw, N, keys, idx, d_err);
    ++launches;
    // the image of every source, its key and its original (src); orig: sorted point -> original
    int* src = nullptr;
    int* orig = nullptr;
    if (padded) {
        void* vorig;
        CKS(ensure(plan, B_SRC, (size_t)N * sizeof(int), &vsrc));
        CKS(ensure(plan, B_ORIG, (size_t)N * sizeof(int), &vorig));
        src = (int*)vsrc;
        orig = (int*)vorig;
        const int* ioff = (const int*)vicnt + N0 + 1;
        k_images<true><<<nblk(N0, 256), 256, 0, st>>>(N0, pts, g, (double*)vw, N, nullptr, ioff, keys, idx, src);
        ++launches;
    }
    int cube_bits = 0;
    while ((1 << cube_bits) < Mtot) ++cube_bits;
    const int end_bit = 3 * kBits + cube_bits;
    void* vcub = nullptr;
    size_t cub_cap = 0;
    const uint64_t* pkeys = keys2;
    // FP32 path: per sorted point a record of the leading/trailing FP32 parts of the
    // coordinates and the FP32 strengths, so that the leaf stage forms source offsets without
    // FP64 arithmetic and reads a source in one piece
    float* pk = nullptr;
    if (sizeof(T) == 4) {
        void* vxf;
        CKS(ensure(plan, B_XF, (size_t)N * point_record_floats(drho) * sizeof(float), &vxf));
        pk = (float*)vxf;
    }
    const int ngb = (int)((N + kGatherThreads - 1) / kGatherThreads);
    void* vpart;
    CKS(ensure(plan, B_PART, (size_t)ngb * 2 * drho * sizeof(double), &vpart));
    int* d_nR = (int*)((char*)vmisc + 1024);       // non-leaf count per level
    int* d_missing = (int*)((char*)vmisc + 1280);  // balance check, per level
    int* d_nleaf = (int*)((char*)vmisc + 1536);
    int* d_next = (int*)((char*)vmisc + 2040);     // residual-task counter of k_pair
    int* d_capped = (int*)((char*)vmisc + 1352);   // depth-cap cells over n_s (after missing[])
    // cells with more than n_s points are disjoint: at most N/(n_s+1) split per level
    const int64_t cap = std::max<int64_t>(1, N / ((int64_t)plan->n_s + 1));
    const int nblkR = (int)((N + kRefineThreads - 1) / kRefineThreads);
    void *vrblk, *vR;
    CKS(ensure(plan, B_CNT, (size_t)2 * kBits * nblkR * sizeof(int), &vrblk));
    CKS(ensure(plan, B_R, (size_t)kBits * cap * sizeof(uint64_t), &vR));
    int* bcnt = (int*)vrblk;
    int* boff = bcnt + (size_t)kBits * nblkR;
    uint64_t* Rall = (uint64_t*)vR;
    // one pinned readback of nR[0..kBits] (misc + 1024) and missing[] (misc + 1280)
    const int* hmeta = (const int*)plan->h_meta;
    const int kMissing = 64;                              // int offset of missing[] in the copy
    // ---- (1)+(2) sort on the leading key bits, gather, one-pass refinement; repeated with all
    // key bits if the forest reaches the sorted depth ----------------------------------------
    // Levels the keys are sorted to first (their leading 3 lsort bits): the depth a forest of
    // N points with n_s per leaf reaches when they are uniform, plus four levels.  Deeper
    // forests (clustered points) sort again on all bits.  The choice depends on N and n_s only,
    // so the point order within a leaf -- and with it the rounding of every sum -- is the same
    // for the same input, whatever the plan evaluated before.
    int lsort = 4;
    for (double cells = (double)N / plan->n_s; cells > 1.0 && lsort < kBits; cells /= 8.0) ++lsort;
    for (int attempt = 0;; ++attempt) {
        const int begin_bit = 3 * (kBits - lsort);
        size_t tmp_bytes = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys, keys2, idx, idx2, (int)N, begin_bit, end_bit, st);
        CKS(ensure(plan, B_CUB, std::max<size_t>(tmp_bytes, 1 << 20), &vcub));
        cub_cap = plan->bufs[B_CUB].cap;
        CK(cub::DeviceRadixSort::SortPairs(vcub, tmp_bytes, keys, keys2, idx, idx2, (int)N, begin_bit, end_bit, st));
        // strength sums over the original points (a shard: over its own points, first n_own)
        k_gather<<<ngb, kGatherThreads, 0, st>>>(N, sh ? sh->n_sum : N0, drho, idx2, src, g, (const double*)vw, rho,
                                                  xs, rs, pk, orig, (double*)vpart);
        k_sum_partials<<<1, 1024, 0, st>>>(ngb, 2 * drho, (const double*)vpart, d_sums);
        CK(cudaMemsetAsync(d_missing, 0, (kBits + 1) * sizeof(int), st));      // missing[] and capped
        k_refine_count<<<nblkR, kRefineThreads, 0, st>>>(N, pkeys, plan->n_s, nblkR, lsort, bcnt, d_capped);
        k_refine_scan<<<1, 1024, 0, st>>>(nblkR, bcnt, boff, d_nR);
        k_refine_write<<<nblkR, kRefineThreads, 0, st>>>(N, pkeys, plan->n_s, nblkR, lsort, boff, cap, Rall);
        {
            const int64_t nchk = (int64_t)(kBits - 1) * 27 * cap;
            k_balance_check<<<(unsigned)((nchk + 255) / 256), 256, 0, st>>>(cap, Rall, d_nR, g, d_missing);
        }
        launches += 11;
        CK(cudaMemcpyAsync(plan->h_meta, d_nR, 512, cudaMemcpyDeviceToHost, st));
        CKS(host_wait(plan, st));
        if (lsort >= kBits || hmeta[lsort - 1] == 0) break;
        lsort = kBits;                                     // deeper than the sorted bits: resort
    }
    const int n_capped = hmeta[(1352 - 1024) / 4];
    TreeInfo ti;
    std::vector<const uint64_t*> Rl(kMaxLevels + 1, nullptr);
    // balance arrays that outgrow the refinement layout: stream-ordered, released on return
    std::vector<void*> level_mem;
    auto alloc_level = [&](size_t bytes, void** out) -> dmk_status_t {
        if (plan->arena) return arena_take(plan, bytes, out);
        void* p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, std::max<size_t>(bytes, 16), st);
        if (e != cudaSuccess) { plan->err = "level allocation failed"; return DMK_ERR_OOM; }
        ++plan->n_allocs;
        level_mem.push_back(p);
        *out = p;
        return DMK_OK;
    };
    auto free_levels = [&]() { for (void* p : level_mem) cudaFreeAsync(p, st); level_mem.clear(); };
    struct Guard { std::function<void()> f; ~Guard() { f(); } };
    Guard guard{free_levels};
    int nlev = kBits + 1;
    for (int k = 0; k <= kBits; ++k)
        if (hmeta[k] == 0) { nlev = k + 1; break; }
    for (int l = 0; l < nlev; ++l) Rl[l] = Rall + (size_t)l * cap;
    bool balanced = true;
    for (int k = 0; k < kBits; ++k)
        if (hmeta[kMissing + k] != 0) balanced = false;
    std::vector<int64_t> cR(nlev);
    for (int k = 0; k < nlev; ++k) cR[k] = hmeta[k];
    // ---- (3) 2:1 balance, finest non-leaf level upward (only when the check found gaps) -----
    // Small levels: one single-CTA kernel per level, no host round trip until the end; if one
    // of them reports more new cells than it holds, the general path below redoes the balance
    // from the refinement arrays.
    bool need_general = false;
    if (!balanced) {
        int64_t worst = 0;
        for (int l = 1; l < nlev; ++l) worst = std::max(worst, 27 * cR[l]);
        if (worst <= ((int64_t)1 << 20)) {
            int* d_overflow = (int*)((char*)vmisc + 1600);
            std::vector<const uint64_t*> Rs(Rl);
            std::vector<int64_t> cs(cR);
            // every level's output from one plan buffer (no allocation per level)
            auto bal_bytes = [&](int l) { return ((size_t)(cR[l - 1] + kBalNew) * sizeof(uint64_t) + 255) & ~(size_t)255; };
            size_t bal_total = 0;
            for (int l = nlev - 2; l >= 1; --l) bal_total += bal_bytes(l);
            void* vbal;
            CKS(ensure(plan, B_BAL, bal_total, &vbal));
            size_t bal_off = 0;
            for (int l = nlev - 2; l >= 1; --l) {
                void* vo = (char*)vbal + bal_off;
                bal_off += bal_bytes(l);
                k_balance_small<<<1, kBalThreads, 0, st>>>(Rs[l], Rs[l - 1], d_nR, l, g, (uint64_t*)vo, d_overflow);
                Rs[l - 1] = (const uint64_t*)vo;
                cs[l - 1] += kBalNew;
                ++launches;
            }
            CK(cudaMemcpyAsync(plan->h_meta, d_nR, 1024, cudaMemcpyDeviceToHost, st));
            CKS(host_wait(plan, st));
            if (hmeta[(1600 - 1024) / 4] == 0) {
                Rl = Rs;
            } else {
                need_general = true;
                // restore the refinement counts
                for (int k = 0; k < nlev; ++k) ((int*)plan->h_meta)[k] = (int)cR[k];
                CK(cudaMemcpyAsync(d_nR, plan->h_meta, nlev * sizeof(int), cudaMemcpyHostToDevice, st));
            }
        } else {
            need_general = true;
        }
    }
    if (need_general) {
        for (int l = nlev - 2; l >= 1; --l) {
            const int64_t capP = cR[l - 1];
            const int64_t ncand = 27 * cR[l] + capP;
            void *va, *vb;
            CKS(alloc_level((size_t)ncand * sizeof(uint64_t), &va));
            CKS(alloc_level((size_t)ncand * sizeof(uint64_t), &vb));
            k_balance_cand<<<nblk(ncand, 256), 256, 0, st>>>((int)cR[l], Rl[l], d_nR + l, (int)capP, Rl[l - 1],
                                                             d_nR + l - 1, l, g, (uint64_t*)va);
            // keys of level l-1 are below Mtot 8^(l-1); one more bit keeps the all-ones padding last
            const int kbits = std::min(64, cube_bits + 3 * (l - 1) + 1);
            size_t tb = 0, tb2 = 0;
            cub::DeviceRadixSort::SortKeys(nullptr, tb, (uint64_t*)va, (uint64_t*)vb, (int)ncand, 0, kbits, st);
            cub::DeviceSelect::Unique(nullptr, tb2, (uint64_t*)vb, (uint64_t*)va, d_nR + l - 1, (int)ncand, st);
            if (std::max(tb, tb2) > cub_cap) { CKS(ensure(plan, B_CUB, std::max(tb, tb2), &vcub)); cub_cap = plan->bufs[B_CUB].cap; }
            CK(cub::DeviceRadixSort::SortKeys(vcub, tb, (uint64_t*)va, (uint64_t*)vb, (int)ncand, 0, kbits, st));
            CK(cub::DeviceSelect::Unique(vcub, tb2, (uint64_t*)vb, (uint64_t*)va, d_nR + l - 1, (int)ncand, st));
            k_trim_invalid<<<1, 1, 0, st>>>((uint64_t*)va, d_nR + l - 1);
            Rl[l - 1] = (const uint64_t*)va;
            const int64_t maxcells = (3 * (l - 1) < 40) ? ((int64_t)Mtot << (3 * (l - 1))) : ncand;
            cR[l - 1] = std::min(ncand, maxcells);
            launches += 6;
        }
        CK(cudaMemcpyAsync(plan->h_meta, d_nR, nlev * sizeof(int), cudaMemcpyDeviceToHost, st));
        CKS(host_wait(plan, st));
    }
    for (int k = 0; k < nlev; ++k) {
        ti.nR.push_back(hmeta[k]);
        ti.ncell.push_back(k == 0 ? Mtot : 8 * hmeta[k - 1]);
    }
    // ---- (4) box arrays -----------------------------------------------------------------
    ti.nlev = nlev;
    ti.off.assign(nlev + 1, 0);
    ti.nl_off.assign(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) {
        ti.off[l + 1] = ti.off[l] + ti.ncell[l];
        ti.nl_off[l + 1] = ti.nl_off[l] + ti.nR[l];
    }
    const int nb = ti.off[nlev], n_nl = ti.nl_off[nlev];
    ti.nb = nb;
    ti.n_nl = n_nl;
    void *vbu, *vbi;
    CKS(ensure(plan, B_BOXU64, (size_t)nb * sizeof(uint64_t), &vbu));
    // layout: level(1) ix(3) start(1) end(1) child0(1) parent(1) nl(1) coll(27) = 36 per box
    CKS(ensure(plan, B_BOXINT, (size_t)nb * 36 * sizeof(int) + 2 * (kMaxLevels + 2) * sizeof(int), &vbi));
    BoxArrays B;
    B.key = (uint64_t*)vbu;
    int* bi = (int*)vbi;
    B.level = bi; B.ix = bi + nb; B.start = bi + 4 * nb; B.end = bi + 5 * nb; B.child0 = bi + 6 * nb;
    B.parent = bi + 7 * nb; B.nl = bi + 8 * nb; B.coll = bi + 9 * nb;
    LevelSet ls;
    std::memset(&ls, 0, sizeof(ls));
    ls.nlev = nlev;
    for (int l = 0; l <= nlev; ++l) {
        ls.off[l] = ti.off[l];
        ls.nl_off[l] = ti.nl_off[l];
    }
    for (int l = 0; l < nlev; ++l) {
        ls.R[l] = Rl[l];
        ls.nR[l] = ti.nR[l];
    }
    void *vnl, *vflags, *vleaves, *viota;
    CKS(ensure(plan, B_NLBOX, (size_t)std::max(n_nl, 1) * sizeof(int), &vnl));
    CKS(ensure(plan, B_FLAGS, (size_t)nb * sizeof(int), &vflags));
    CKS(ensure(plan, B_LEAVES, (size_t)nb * sizeof(int), &vleaves));
    CKS(ensure(plan, B_CAND, (size_t)nb * sizeof(int), &viota));
    int* nl_box = (int*)vnl;
    int* leaves = (int*)vleaves;
    k_box_fill_all<<<nblk(nb, 256), 256, 0, st>>>(ls, nb, pkeys, N, g, B, nl_box, (int*)vflags, (int*)viota);
    k_colleagues<<<nblk((int64_t)27 * nb, 256), 256, 0, st>>>(nb, B.level, B.ix, B.key, ls, g, B.coll);
    launches += 2;
    // leaves with points, in box order
    {
        size_t tb = 0;
        cub::DeviceSelect::Flagged(nullptr, tb, (int*)viota, (int*)vflags, leaves, d_nleaf, nb, st);
        if (tb > cub_cap) { CKS(ensure(plan, B_CUB, tb, &vcub)); cub_cap = plan->bufs[B_CUB].cap; }
        CK(cub::DeviceSelect::Flagged(vcub, tb, (int*)viota, (int*)vflags, leaves, d_nleaf, nb, st));
        launches += 2;
    }
    // direct lists and residual tasks: counts for every possible leaf slot (entries in the
    // first nb + 1 ints, tasks in the next nb + 1), one scan over both, one readback of the totals
    void *vdo, *vdl, *vtk;
    CKS(ensure(plan, B_DOFFS, 2 * (size_t)(nb + 1) * sizeof(int), &vdo));
    int* doffs = (int*)vdo;
    int* toffs = doffs + nb + 1;
    CK(cudaMemsetAsync(doffs, 0, 2 * (size_t)(nb + 1) * sizeof(int), st));
    k_direct<false><<<nblk((int64_t)32 * nb, 128), 128, 0, st>>>(nb, d_nleaf, leaves, B, g, doffs, nullptr, nullptr,
                                                                 d_pairs, nb + 1, nullptr);
    {
        size_t tb = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, tb, doffs, doffs, 2 * (nb + 1), st);
        if (tb > cub_cap) { CKS(ensure(plan, B_CUB, tb, &vcub)); cub_cap = plan->bufs[B_CUB].cap; }
        CK(cub::DeviceScan::ExclusiveSum(vcub, tb, doffs, doffs, 2 * (nb + 1), st));
        // pinned readback: misc + 768 .. + 1540 holds the pair count and the leaf count; read by
        // the host only after the upward pass is queued (ev_cnt), so the GPU does not wait for it
        CK(cudaMemcpyAsync(plan->h_meta, (char*)vmisc + 768, 772, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(plan->h_meta + 1024, doffs + nb, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(plan->ev_cnt, st));
        launches += 3;
    }
    // leaf boxes (with or without points): the bound used before the leaf count is read back
    const int nleaf_cap = nb - n_nl;
    int nleaf = 0;
    DirectEntry* dl = nullptr;
    int4* tasks = nullptr;
    rec(1);
    // ---- leaf residual sums: they need only the tree, so with pair_overlap they run on the
    // side stream beside the far field (steps 5-8) and are joined before the leaf expansions
    LeafOut lo;
    lo.pot = pot;
    lo.grad = grad;
    lo.perm = idx2;
    lo.orig = orig ? orig : idx2;
    lo.n_orig = sh ? sh->n_out : N0;
    lo.rs = rs;
    lo.self_val = plan->d_self;
    lo.self_grad = plan->d_self + P.d_u * P.d_rho;
    lo.pk = reinterpret_cast<const float4*>(pk);
    // the truncated-kernel constants, formed after the root stage (k_root_const)
    double* d_ucst = (double*)((char*)vmisc + 1664);
    lo.ucst = d_ucst;
    const bool gr = grad != nullptr;
    bool fast_leaf = false, overlap = false;
    auto run_pair = [&](cudaStream_t sp) -> dmk_status_t {
        if (plan->timing) cudaEventRecord(plan->ev[8], sp);
        switch (P.kernel) {
            case DMK_LAPLACE: CKS((gr ? launch_pair<T, DMK_LAPLACE, true> : launch_pair<T, DMK_LAPLACE, false>)(plan, tab, leaves, B, xs, N, doffs, dl, lo, toffs, nb, tasks, d_next, sp)); break;
            case DMK_STOKESLET: CKS((gr ? launch_pair<T, DMK_STOKESLET, true> : launch_pair<T, DMK_STOKESLET, false>)(plan, tab, leaves, B, xs, N, doffs, dl, lo, toffs, nb, tasks, d_next, sp)); break;
            case DMK_STRESSLET: CKS((gr ? launch_pair<T, DMK_STRESSLET, true> : launch_pair<T, DMK_STRESSLET, false>)(plan, tab, leaves, B, xs, N, doffs, dl, lo, toffs, nb, tasks, d_next, sp)); break;
            default: CKS((gr ? launch_pair<T, DMK_ROTLET, true> : launch_pair<T, DMK_ROTLET, false>)(plan, tab, leaves, B, xs, N, doffs, dl, lo, toffs, nb, tasks, d_next, sp)); break;
        }
        if (plan->timing) cudaEventRecord(plan->ev[9], sp);
        ++launches;
        return DMK_OK;
    };
    // the direct lists' counts (queued before the upward pass), the filled lists and tasks, and
    // with pair_overlap the residual sums on the side stream, which waits for the counts only
    auto finish_direct = [&]() -> dmk_status_t {
        CKS(host_wait_event(plan, plan->ev_cnt));
        int n_entries = 0;
        std::memcpy(&ti.n_pairs, plan->h_meta, sizeof(unsigned long long));
        std::memcpy(&ti.n_leafp, plan->h_meta + (1536 - 768), sizeof(int));
        std::memcpy(&n_entries, plan->h_meta + 1024, sizeof(int));
        ti.n_entries = n_entries;
        nleaf = ti.n_leafp;
        fast_leaf = nleaf > 0 && p <= kMaxPFast;
        overlap = fast_leaf && plan->pair_overlap;
        CKS(ensure(plan, B_DL, (size_t)std::max<int64_t>(ti.n_entries, 1) * sizeof(DirectEntry), &vdl));
        dl = (DirectEntry*)vdl;
        // at most nt / kPairTile + kPairTileLog tasks per leaf
        CKS(ensure(plan, B_TASKS, ((size_t)N / kPairTile + (size_t)kPairTileLog * nleaf + 1) * sizeof(int4), &vtk));
        tasks = (int4*)vtk;
        const cudaStream_t sd = overlap ? plan->side : st;
        if (overlap) CK(cudaStreamWaitEvent(plan->side, plan->ev_cnt, 0));
        if (nleaf > 0)
            k_direct<true><<<nblk((int64_t)32 * nleaf, 128), 128, 0, sd>>>(nleaf, d_nleaf, leaves, B, g, nullptr,
                                                                           doffs, dl, nullptr, nb + 1, tasks);
        ++launches;
        if (overlap) {
            CKS(run_pair(plan->side));
            CK(cudaEventRecord(plan->ev_join, plan->side));
        }
        return DMK_OK;
    };
    // ---- (5) upward pass ---------------------------------------------------------------
    void *vpr, *vloc;
    CKS(ensure(plan, B_PROXY, (size_t)nb * drho * p3 * sizeof(T), &vpr));
    CKS(ensure(plan, B_LOCAL, (size_t)nb * du * p3 * sizeof(T), &vloc));
    T* proxy = (T*)vpr;
    T* local = (T*)vloc;
    // FP32 path, p <= 24 (direct_leaf): the leaf sources go straight onto the parent grids
    // (k_anterp3), every proxy that is read (non-leaf boxes, cubes) written by it, by
    // k_leaf_partials or by the upward pass over the non-leaf children; the leaf targets
    // evaluate their parent's expansion (downward).  Otherwise leaf proxies, the upward pass
    // over all children, and a zeroed array.
    //   The direct upward work goes by parents (one item per parent of leaves) when they are
    // enough work items for the GPU, else split by leaves (split_up: each leaf onto its
    // parent's grid in its own slot, then summed per parent in child order)
    const bool direct_leaf = sizeof(T) == 4 && p <= 24;
    const bool direct_up = direct_leaf;
    const bool split_up = direct_leaf && n_nl + Mtot < 2 * plan->n_sm;
    if (!direct_up) {
        CK(cudaMemsetAsync(proxy, 0, (size_t)nb * drho * p3 * sizeof(T), st));
        ++launches;
    }
    CK(cudaMemsetAsync(local, 0, (size_t)nb * du * p3 * sizeof(T), st));
    ++launches;
    bool anterp_done = false;
    if constexpr (sizeof(T) == 4) {
        if (direct_leaf && nleaf_cap > 0) {
            const int items = split_up ? nleaf_cap : n_nl + Mtot;
            const unsigned grid = (unsigned)std::max(1, std::min(items, plan->n_sm * 8));
            const int TN = p <= 20 ? 20 : 24;
            const int ntile = drho * ((p + 3) / 4) * p * ((p + TN - 1) / TN);
            const int threads = std::min(kAntThreads, (ntile + 31) / 32 * 32);
            auto launch = [&](auto kern, size_t sm) -> dmk_status_t {
                CKS(set_smem(plan, kern, sm));
                kern<<<grid, threads, sm, st>>>(n_nl, nl_box, Mtot, B, xs, N, rs, tab, plan->T.s, (float*)proxy,
                                                split_up ? leaves : nullptr, d_nleaf, 1);
                return DMK_OK;
            };
            if (p <= 20) {
                if (split_up) CKS(launch(k_anterp3<20, 20, kAntRowsLeaf>, anterp3_smem<20>(true)));
                else CKS(launch(k_anterp3<20, 20, kAntRows>, anterp3_smem<20>(false)));
            } else {
                if (split_up) CKS(launch(k_anterp3<24, 24, kAntRowsLeaf>, anterp3_smem<24>(true)));
                else CKS(launch(k_anterp3<24, 24, kAntRows>, anterp3_smem<24>(false)));
            }
            ++launches;
            if (split_up && n_nl > 0) {
                const int per_box = drho * p3;
                k_leaf_partials<float><<<nblk((int64_t)n_nl * per_box, 256), 256, 0, st>>>(n_nl, nl_box, B, per_box,
                                                                                         (float*)proxy);
                ++launches;
            }
            anterp_done = true;
        }
    }
    if (nleaf_cap > 0 && !anterp_done) {
        if (p <= 20) CKS((launch_anterp2<T, 20>(plan, tab, nleaf_cap, d_nleaf, leaves, B, xs, N, rs, proxy)));
        else if (p <= 24) CKS((launch_anterp2<T, 24>(plan, tab, nleaf_cap, d_nleaf, leaves, B, xs, N, rs, proxy)));
        else CKS((launch_anterp<T, 48>(plan, tab, nleaf_cap, d_nleaf, leaves, B, xs, N, rs, proxy)));
        ++launches;
    }
    Evaluator<T> ev(plan, tab);
    const int pitch = odd_pitch(p);
    const int up_threads = (((p * p + 1) / 2 + 31) / 32) * 32;     // k_up_cluster: two fibers per thread
    const int shift_threads = ((p * p + 31) / 32) * 32;            // k_shift_child: one fiber per thread
    const int mp = (p <= 20) ? 20 : kMaxPFast;     // register width of the fiber kernels
    // per-child tensor kernels: three operators and two padded p^3 buffers per CTA
    const size_t ch_bytes = (3 * (size_t)mp * mp + 2 * (size_t)p * p * pitch) * sizeof(T);
    const bool fast_up = p <= kMaxPFast && ch_bytes <= plan->smem_optin;
    const bool fast_shift = fast_up;
    if (direct_leaf && !fast_up) { plan->err = "internal: the cluster upward pass does not fit"; return DMK_ERR_CUDA; }
    if (fast_up) {
        if (mp == 20) CKS(set_smem(plan, k_up_cluster<T, 20>, ch_bytes));
        else CKS(set_smem(plan, k_up_cluster<T, kMaxPFast>, ch_bytes));
    }
    for (int l = nlev - 2; l >= 0; --l) {
        const int n = ti.nR[l];
        if (n == 0) continue;
        // direct path: parents whose children are all leaves have their proxies already
        if (direct_up && ti.nR[l + 1] == 0) continue;
        if (fast_up) {
            if (mp == 20)
                k_up_cluster<T, 20><<<8 * n, up_threads, ch_bytes, st>>>(nl_box + ti.nl_off[l], B, tab, proxy,
                                                                        direct_up ? 1 : 0);
            else
                k_up_cluster<T, kMaxPFast><<<8 * n, up_threads, ch_bytes, st>>>(nl_box + ti.nl_off[l], B, tab,
                                                                               proxy, direct_up ? 1 : 0);
        } else {
            Place pl;
            unsigned char* scr;
            size_t bytes = 3 * (size_t)p3 * sizeof(T);
            CKS(ev.place(bytes, n, pl, &scr));
            CKS(set_smem(plan, k_upward<T>, pl.use_smem ? bytes : 0));
            k_upward<T><<<pl.grid, 256, pl.use_smem ? bytes : 0, st>>>(n, nl_box + ti.nl_off[l], B, tab, proxy, scr,
                                                                      bytes, pl.use_smem);
        }
        ++launches;
    }
    rec(2);
    CKS(finish_direct());
    // ---- (6) root far field (FP64) ----------------------------------------------------------
    {
        const RootTab& rt = plan->root;
        // the second part (original symbol for alpha != 0, App. E switch), if any
        const RootTab& rt2 = plan->root2;
        const int nparts = rt2.nmode > 0 ? 2 : 1;
        const int nmode_max = std::max(rt.nmode, rt2.nmode);
        // sums over the cubes as DFTs over the cube index (Sec. 3.4, 5.4) where the plan admits them
        const bool dft_root = P.root_dft;
        void *vchi, *vuh, *vrsc;
        CKS(ensure(plan, B_CHI, (size_t)(dft_root ? 1 : Mtot) * drho * (rt.nmode + rt2.nmode) * sizeof(Cx<double>),
                   &vchi));
        CKS(ensure(plan, B_UHAT, (size_t)du * nmode_max * sizeof(Cx<double>), &vuh));
        const int jf = Mtot * drho, jb = Mtot * du;
        // scratch of the direct sums: forward B1 (n1 p^2) + B2 (n1 n2 p) per (cube, strength
        // component); backward G (nmode) + C2 (n1 n2 p) + C1 (n1 p^2) per (cube, potential
        // component).  Of the DFTs: forward B1 and B2 per (cube, component), the sums over m1, m2
        // (M3 n1 n2 p) and the transform (Q3 n1 n2 p) per component; backward C2 (Q3 n1 n2 p) and
        // Dm (M3 n1 n2 p) per component, C1 per (cube, component)
        size_t nscr = 0;
        for (int ip = 0; ip < nparts; ++ip) {
            const RootTab& r = ip == 0 ? rt : rt2;
            const size_t h1 = (size_t)r.n1 * p * p, h2 = (size_t)r.n1 * r.n2 * p;
            if (dft_root) {
                const size_t M3 = (size_t)g.M[2], Q3 = (size_t)r.Q[2];
                nscr = std::max(nscr, (size_t)jf * (h1 + h2) + (M3 + Q3) * drho * h2);
                nscr = std::max(nscr, (Q3 + M3) * du * h2 + (size_t)jb * h1);
            } else {
                nscr = std::max(nscr, std::max((size_t)jf * (h1 + h2), (size_t)jb * (r.nmode + h2 + h1)));
            }
        }
        CKS(ensure(plan, B_SCRATCH, nscr * sizeof(Cx<double>), &vrsc));
        Cx<double>* r0 = (Cx<double>*)vrsc;
        Cx<double>* chi = (Cx<double>*)vchi;
        Cx<double>* uh = (Cx<double>*)vuh;
        auto blocks = [](int64_t n) { return (unsigned)((n + 127) / 128); };
        // the root proxies of the structure factor: a non-exact tiling counts only the sources
        // inside Omega (cube proxies inside, nothing for padding cubes, cut cubes from their
        // original sources)
        const T* rproxy = proxy;
        const bool owned_only = sh && sh->cube_owned;
        if (padded || owned_only) {
            void* vchip;
            CKS(ensure(plan, B_CHIP, (size_t)Mtot * drho * p3 * sizeof(T), &vchip));
            T* chip = (T*)vchip;
            const int* cls = plan->d_cube;
            if (owned_only) {
                // a shard: the cubes it owns count (class 0), the others not (class 2)
                void* vcls;
                CKS(ensure(plan, B_SHARDCLS, (size_t)Mtot * sizeof(int), &vcls));
                std::vector<int> hc(Mtot);
                for (int m = 0; m < Mtot; ++m) hc[m] = sh->cube_owned[m] ? 0 : 2;
                CK(cudaMemcpyAsync(vcls, hc.data(), Mtot * sizeof(int), cudaMemcpyHostToDevice, st));
                CK(cudaStreamSynchronize(st));
                cls = (const int*)vcls;
            }
            k_chi_proxy<T><<<nblk((int64_t)Mtot * drho * p3, 256), 256, 0, st>>>(Mtot, drho, p3, cls, proxy, chip);
            const int ncut = owned_only ? 0 : (int)std::count(P.cube_class.begin(), P.cube_class.end(), 1);
            if (ncut > 0) {
                const int* cutlist = plan->d_cube + Mtot + 1;
                if (p <= 20) {
                    const int threads = (20 * 20 + 31) / 32 * 32;
                    const size_t sm = 3 * (size_t)kAnterpChunk * 20 * sizeof(T);
                    CKS(set_smem(plan, k_anterp<T, 20>, sm));
                    k_anterp<T, 20><<<ncut, threads, sm, st>>>(plan->d_cube + Mtot, cutlist, B, xs, N, rs, tab, P.s,
                                                              chip, idx2, N0);
                } else if (p <= 24) {
                    const int threads = (24 * 24 + 31) / 32 * 32;
                    const size_t sm = 3 * (size_t)kAnterpChunk * 24 * sizeof(T);
                    CKS(set_smem(plan, k_anterp<T, 24>, sm));
                    k_anterp<T, 24><<<ncut, threads, sm, st>>>(plan->d_cube + Mtot, cutlist, B, xs, N, rs, tab, P.s,
                                                              chip, idx2, N0);
                } else {
                    const size_t sm = 3 * (size_t)kAnterpChunk * 48 * sizeof(T);
                    CKS(set_smem(plan, k_anterp<T, 48>, sm));
                    k_anterp<T, 48><<<ncut, 512, sm, st>>>(plan->d_cube + Mtot, cutlist, B, xs, N, rs, tab, P.s, chip,
                                                          idx2, N0);
                }
                ++launches;
            }
            rproxy = chip;
            ++launches;
        }
        const RootTab* parts[2] = {&rt, &rt2};
        if (dft_root) {
            // per part: chi of all cubes as one (part 1 after part 0), one reduction of both
            // (sharded evaluations), then the evaluation; part 1 adds to part 0
            const int M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
            Cx<double>* chis[2] = {chi, chi + (size_t)drho * rt.nmode};
            for (int ip = 0; ip < nparts; ++ip) {
                const RootTab& r = *parts[ip];
                const size_t h1 = (size_t)r.n1 * p * p, h2 = (size_t)r.n1 * r.n2 * p;
                Cx<double>* B1f = r0;
                Cx<double>* B2f = B1f + (size_t)jf * h1;
                Cx<double>* Af = B2f + (size_t)jf * h2;
                Cx<double>* Bh = Af + (size_t)M3 * drho * h2;
                k_root_fwd1<T><<<blocks((int64_t)jf * h1), 128, 0, st>>>(jf, p, r, rproxy, B1f);
                k_root_fwd2<<<blocks((int64_t)jf * h2), 128, 0, st>>>(jf, p, r, B1f, B2f);
                const Cx<double>* a3 = B2f;
                if (M1 * M2 > 1) {
                    k_rootdft_fold12<<<blocks((int64_t)M3 * drho * h2), 128, 0, st>>>(M1, M2, M3, drho, p, r, B2f,
                                                                                        Af);
                    a3 = Af;
                    ++launches;
                }
                k_rootdft_fwd3<<<blocks((int64_t)r.Q[2] * drho * h2), 128, 0, st>>>(M3, drho, (int)h2, r, a3, Bh);
                k_rootdft_chi<<<blocks((int64_t)drho * r.nmode), 128, 0, st>>>(drho, p, g, r, Bh, chis[ip]);
                launches += 4;
            }
            CKS(reduce_chi(plan, sh, chi, (int64_t)2 * drho * (rt.nmode + rt2.nmode), d_sums));
            for (int ip = 0; ip < nparts; ++ip) {
                const RootTab& r = *parts[ip];
                const size_t h1 = (size_t)r.n1 * p * p, h2 = (size_t)r.n1 * r.n2 * p;
                k_root_apply<<<nblk(r.nmode, 128), 128, 0, st>>>(1, drho, du, r, chis[ip], uh);
                Cx<double>* C2 = r0;
                Cx<double>* Dm = C2 + (size_t)r.Q[2] * du * h2;
                Cx<double>* C1 = Dm + (size_t)M3 * du * h2;
                k_rootdft_bwd1<<<blocks((int64_t)r.Q[2] * du * h2), 128, 0, st>>>(du, p, g, r, uh, C2);
                k_rootdft_idft3<<<blocks((int64_t)M3 * du * h2), 128, 0, st>>>(M3, du, (int)h2, r, C2, Dm);
                k_rootdft_bwd2<<<blocks((int64_t)jb * h1), 128, 0, st>>>(Mtot, du, p, g, r, Dm, C1);
                k_rootdft_bwd3<T><<<blocks((int64_t)jb * p * p * p), 128, 0, st>>>(Mtot, du, p, g, r, C1, local, ip);
                launches += 5;
            }
        } else {
        // per part: structure factor of every cube (chi of part 1 after that of part 0), one
        // reduction of both (sharded evaluations), then the evaluation; part 1 adds to part 0
        Cx<double>* chis[2] = {chi, chi + (size_t)Mtot * drho * rt.nmode};
        for (int ip = 0; ip < nparts; ++ip) {
            const RootTab& r = *parts[ip];
            const size_t h1 = (size_t)r.n1 * p * p, h2 = (size_t)r.n1 * r.n2 * p;
            k_root_fwd1<T><<<blocks((int64_t)jf * h1), 128, 0, st>>>(jf, p, r, rproxy, r0);
            k_root_fwd2<<<blocks((int64_t)jf * h2), 128, 0, st>>>(jf, p, r, r0, r0 + (size_t)jf * h1);
            k_root_fwd3<<<blocks((int64_t)jf * r.nmode), 128, 0, st>>>(jf, drho, p, g, r, r0 + (size_t)jf * h1,
                                                                        chis[ip]);
            launches += 3;
        }
        CKS(reduce_chi(plan, sh, chi, (int64_t)2 * Mtot * drho * (rt.nmode + rt2.nmode), d_sums));
        for (int ip = 0; ip < nparts; ++ip) {
            const RootTab& r = *parts[ip];
            const size_t h1 = (size_t)r.n1 * p * p, h2 = (size_t)r.n1 * r.n2 * p;
            k_root_apply<<<nblk(r.nmode, 128), 128, 0, st>>>(Mtot, drho, du, r, chis[ip], uh);
            Cx<double>* G = r0;
            Cx<double>* C2 = G + (size_t)jb * r.nmode;
            Cx<double>* C1 = C2 + (size_t)jb * h2;
            k_root_bwd0<<<blocks((int64_t)jb * r.nmode), 128, 0, st>>>(jb, du, g, r, uh, G);
            k_root_bwd1<<<blocks((int64_t)jb * h2), 128, 0, st>>>(jb, p, r, G, C2);
            k_root_bwd2<<<blocks((int64_t)jb * h1), 128, 0, st>>>(jb, p, r, C2, C1);
            k_root_bwd3<T><<<blocks((int64_t)jb * p * p * p), 128, 0, st>>>(jb, du, p, r, C1, nullptr, drho, local,
                                                                             ip);
            launches += 5;
        }
        }
    }
    k_root_const<<<1, 32, 0, st>>>(du, drho, plan->root.rconst, d_sums, d_ucst);
    ++launches;
    rec(3);
    // ---- (7) plane waves: outgoing for all non-leaf boxes, then translation + incoming ------
    if (n_nl > 0) {
        const int NF = P.NF, nfh = P.nfh;
        const size_t nW = (size_t)NF * NF * nfh;
        void* vpw;
        CKS(ensure(plan, B_PW, (size_t)n_nl * drho * nW * sizeof(Cx<T>), &vpw));
        Cx<T>* W = (Cx<T>*)vpw;
        // outgoing transform with the node and mode symmetries (k_pwout3) when its arrays fit in
        // shared memory (the range of |m2| split in parts if needed), else the generic kernel
        const int MH = nfh <= 16 ? 16 : (nfh <= 20 ? 20 : 0);
        bool pwout_done = false;
        if (p <= kMaxPFast && MH > 0) {
            int nsplit = 1;
            while (nsplit < nfh && pwout3_smem<T>(p, nfh, MH, nsplit) > plan->smem_optin) ++nsplit;
            const size_t po3 = pwout3_smem<T>(p, nfh, MH, nsplit);
            if (po3 <= plan->smem_optin) {
                const unsigned grid = (unsigned)std::min<int64_t>((int64_t)nsplit * n_nl, (int64_t)plan->n_sm * 2);
                if (MH == 16) {
                    CKS(set_smem(plan, k_pwout3<T, 16>, po3));
                    k_pwout3<T, 16><<<grid, pw_sym_threads<T>(), po3, st>>>(n_nl, nl_box, tab, proxy, W, nsplit);
                } else {
                    CKS(set_smem(plan, k_pwout3<T, 20>, po3));
                    k_pwout3<T, 20><<<grid, pw_sym_threads<T>(), po3, st>>>(n_nl, nl_box, tab, proxy, W, nsplit);
                }
                ++launches;
                pwout_done = true;
            }
        }
        if (!pwout_done) {
            size_t bytes = ((size_t)p * p * nfh + (size_t)p * NF * nfh) * sizeof(Cx<T>);
            Place pl;
            unsigned char* scr;
            CKS(ev.place(bytes, n_nl, pl, &scr));
            CKS(set_smem(plan, k_pwout<T>, pl.use_smem ? bytes : 0));
            k_pwout<T><<<pl.grid, 256, pl.use_smem ? bytes : 0, st>>>(n_nl, nl_box, tab, proxy, W, scr, bytes,
                                                                     pl.use_smem);
            ++launches;
        }
        rec(4);
        const size_t pw4_bytes = MH > 0 ? pwin4_smem<T>(p, NF, nfh, MH) : 0;
        if (p <= kMaxPFast && MH > 0 && pw4_bytes <= plan->smem_optin) {
            void* vvw;
            CKS(ensure(plan, B_VW, (size_t)n_nl * du * nW * sizeof(Cx<T>), &vvw));
            Cx<T>* Vw = (Cx<T>*)vvw;
            const int nchunk = (int)((nW + kTransThreads - 1) / kTransThreads);
            const unsigned tgrid = (unsigned)(((nchunk + kTransGroup - 1) / kTransGroup) * (int64_t)n_nl * kTransGroup);
            if (drho == 1) {
                k_pw_trans<T, 1, true><<<tgrid, kTransThreads, 0, st>>>(n_nl, nl_box, B, tab, W, 1, Vw);
            } else if (drho == 3) {
                k_pw_trans<T, 3, true><<<tgrid, kTransThreads, 0, st>>>(n_nl, nl_box, B, tab, W, 3, Vw);
            } else {
                k_pw_symbol<T, 9><<<nblk((int64_t)n_nl * nW, kTransThreads), kTransThreads, 0, st>>>(n_nl, nl_box, B,
                                                                                                   tab, W);
                k_pw_trans<T, 3, false><<<tgrid, kTransThreads, 0, st>>>(n_nl, nl_box, B, tab, W, drho, Vw);
                ++launches;
            }
            const unsigned grid = (unsigned)std::min<int64_t>(n_nl, (int64_t)plan->n_sm * 2);
            if (MH == 16) {
                CKS(set_smem(plan, k_pwin4<T, 16>, pw4_bytes));
                k_pwin4<T, 16><<<grid, pw_sym_threads<T>(), pw4_bytes, st>>>(n_nl, nl_box, tab, Vw, local);
            } else {
                CKS(set_smem(plan, k_pwin4<T, 20>, pw4_bytes));
                k_pwin4<T, 20><<<grid, pw_sym_threads<T>(), pw4_bytes, st>>>(n_nl, nl_box, tab, Vw, local);
            }
            launches += 2;
        } else {
            size_t bytes = ((size_t)du * nW + (size_t)p * NF * nfh + (size_t)p * p * nfh) * sizeof(Cx<T>);
            Place pl;
            unsigned char* scr;
            CKS(ev.place(bytes, n_nl, pl, &scr));
            CKS(set_smem(plan, k_pwin<T>, pl.use_smem ? bytes : 0));
            k_pwin<T><<<pl.grid, 256, pl.use_smem ? bytes : 0, st>>>(n_nl, nl_box, B, tab, W, local, scr, bytes,
                                                                    pl.use_smem);
            ++launches;
        }
    } else {
        rec(4);
    }
    rec(5);
    // ---- (8) shift to children, level by level --------------------------------------------
    if (fast_shift) {
        if (mp == 20) CKS(set_smem(plan, k_shift_child<T, 20>, ch_bytes));
        else CKS(set_smem(plan, k_shift_child<T, kMaxPFast>, ch_bytes));
    }
    for (int l = 0; l < nlev - 1; ++l) {
        const int n = ti.nR[l];
        if (n == 0) continue;
        // direct path: leaf children take their parent's expansion, so a level whose children
        // are all leaves has nothing to shift
        if (direct_leaf && ti.nR[l + 1] == 0) continue;
        if (fast_shift) {
            if (mp == 20)
                k_shift_child<T, 20><<<8 * n, shift_threads, ch_bytes, st>>>(nl_box + ti.nl_off[l], B, tab, local,
                                                                            direct_leaf ? 1 : 0);
            else
                k_shift_child<T, kMaxPFast><<<8 * n, shift_threads, ch_bytes, st>>>(nl_box + ti.nl_off[l], B, tab,
                                                                                   local, direct_leaf ? 1 : 0);
        } else {
            Place pl;
            unsigned char* scr;
            size_t bytes = 2 * (size_t)p3 * sizeof(T);
            CKS(ev.place(bytes, n, pl, &scr));
            CKS(set_smem(plan, k_shift<T>, pl.use_smem ? bytes : 0));
            k_shift<T><<<pl.grid, 256, pl.use_smem ? bytes : 0, st>>>(n, nl_box + ti.nl_off[l], B, tab, local, scr,
                                                                     bytes, pl.use_smem);
        }
        ++launches;
    }
    // direct_leaf: the non-leaf boxes with leaf children turn their grids into Chebyshev
    // coefficients (their leaf children's targets evaluate them)
    if (direct_leaf && n_nl > 0) {
        const size_t cb = ((size_t)mp * mp + 2 * (size_t)p * p * pitch) * sizeof(T);
        if (mp == 20) {
            CKS(set_smem(plan, k_box_coef<T, 20>, cb));
            k_box_coef<T, 20><<<n_nl, shift_threads, cb, st>>>(nl_box, B, tab, local);
        } else {
            CKS(set_smem(plan, k_box_coef<T, kMaxPFast>, cb));
            k_box_coef<T, kMaxPFast><<<n_nl, shift_threads, cb, st>>>(nl_box, B, tab, local);
        }
        ++launches;
    }
    // direct_leaf: chunks of targets per item for k_leafexp_parent (counts, exclusive scan)
    int* item_off = nullptr;
    if (direct_leaf) {
        const int n_items = n_nl + Mtot;
        void* vit;
        CKS(ensure(plan, B_ITEMS, (size_t)2 * (n_items + 1) * sizeof(int), &vit));
        int* cnt = (int*)vit;
        item_off = cnt + n_items + 1;
        k_item_chunks<<<nblk(n_items + 1, 256), 256, 0, st>>>(n_nl, nl_box, Mtot, B, cnt);
        size_t tb = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt, item_off, n_items + 1, st);
        if (tb > cub_cap) { CKS(ensure(plan, B_CUB, tb, &vcub)); cub_cap = plan->bufs[B_CUB].cap; }
        CK(cub::DeviceScan::ExclusiveSum(vcub, tb, cnt, item_off, n_items + 1, st));
        launches += 2;
    }
    // leaf grids that did not pass through k_shift_child become Chebyshev coefficients here
    if (nleaf > 0) {
        const int root_only = fast_shift ? 1 : 0;
        const int n = root_only ? std::min(nleaf, Mtot) : nleaf;
        Place pl;
        unsigned char* scr;
        size_t bytes = 2 * (size_t)p3 * sizeof(T);
        CKS(ev.place(bytes, n, pl, &scr));
        CKS(set_smem(plan, k_grid2coef<T>, pl.use_smem ? bytes : 0));
        k_grid2coef<T><<<pl.grid, 256, pl.use_smem ? bytes : 0, st>>>(n, d_nleaf, leaves, B.level, root_only, tab, local, scr,
                                                                      bytes, pl.use_smem);
        ++launches;
    }
    rec(6);
    // ---- (9) leaf stage -----------------------------------------------------------------
    if (fast_leaf) {
        if (overlap) CK(cudaStreamWaitEvent(st, plan->ev_join, 0));
        else CKS(run_pair(st));
        if (plan->timing) cudaEventRecord(plan->ev[10], st);
        switch (P.kernel) {
            case DMK_LAPLACE: CKS((gr ? launch_leafexp<T, DMK_LAPLACE, true> : launch_leafexp<T, DMK_LAPLACE, false>)(plan, tab, nleaf, leaves, B, local, xs, N, lo, direct_leaf ? 1 : 0, n_nl, nl_box, Mtot, item_off)); break;
            case DMK_STOKESLET: CKS((gr ? launch_leafexp<T, DMK_STOKESLET, true> : launch_leafexp<T, DMK_STOKESLET, false>)(plan, tab, nleaf, leaves, B, local, xs, N, lo, direct_leaf ? 1 : 0, n_nl, nl_box, Mtot, item_off)); break;
            case DMK_STRESSLET: CKS((gr ? launch_leafexp<T, DMK_STRESSLET, true> : launch_leafexp<T, DMK_STRESSLET, false>)(plan, tab, nleaf, leaves, B, local, xs, N, lo, direct_leaf ? 1 : 0, n_nl, nl_box, Mtot, item_off)); break;
            default: CKS((gr ? launch_leafexp<T, DMK_ROTLET, true> : launch_leafexp<T, DMK_ROTLET, false>)(plan, tab, nleaf, leaves, B, local, xs, N, lo, direct_leaf ? 1 : 0, n_nl, nl_box, Mtot, item_off)); break;
        }
        ++launches;
    } else if (nleaf > 0) {
        switch (P.kernel) {
            case DMK_LAPLACE: CKS((launch_leaf<T, DMK_LAPLACE>(plan, tab, nleaf, leaves, B, local, xs, N, doffs, dl, lo, gr))); break;
            case DMK_STOKESLET: CKS((launch_leaf<T, DMK_STOKESLET>(plan, tab, nleaf, leaves, B, local, xs, N, doffs, dl, lo, gr))); break;
            case DMK_STRESSLET: CKS((launch_leaf<T, DMK_STRESSLET>(plan, tab, nleaf, leaves, B, local, xs, N, doffs, dl, lo, gr))); break;
            default: CKS((launch_leaf<T, DMK_ROTLET>(plan, tab, nleaf, leaves, B, local, xs, N, doffs, dl, lo, gr))); break;
        }
        ++launches;
    }
    rec(7);
    CK(cudaGetLastError());
    int herr = 0;
    double hs[18];
    // pinned readback of the error flags (misc + 0) and strength sums (misc + 256)
    CK(cudaMemcpyAsync(plan->h_meta, vmisc, 256 + 2 * drho * sizeof(double), cudaMemcpyDeviceToHost, st));
    CKS(host_wait(plan, st));
    std::memcpy(&herr, plan->h_meta, sizeof(int));
    std::memcpy(hs, plan->h_meta + 256, 2 * drho * sizeof(double));
    if (herr & kErrNonFinite) { plan->err = "non-finite coordinate"; return DMK_ERR_OUT_OF_DOMAIN; }
    if (herr & kErrDomain) { plan->err = "a free coordinate lies outside [0, L_i)"; return DMK_ERR_OUT_OF_DOMAIN; }
    if (!plan->allow_charged && !(sh && sh->reduce) && P.kernel == DMK_LAPLACE && (P.D == 1 || P.D == 2) &&
        std::fabs(hs[0]) > 1e-12 * std::max(hs[1], 1e-300)) {
        plan->err = "Laplace with D = 1, 2 requires zero net charge";
        return DMK_ERR_NOT_NEUTRAL;
    }
    if (herr & kErrIndex) { plan->err = "internal index check failed"; return DMK_ERR_CUDA; }
    // stats
    dmk_stats_t& S = plan->stats;
    S.c_times_1000 = (int)std::lround(P.c * 1000);
    S.p = P.p;
    S.n_f = P.nf;
    S.n_root_modes = P.n_root_modes;
    S.n_levels = nlev;
    S.n_boxes = nb;
    S.n_nonleaf = n_nl;
    S.n_leaves = nb - n_nl;
    S.n_pairs = (int64_t)ti.n_pairs;
    S.n_direct_entries = ti.n_entries;
    S.kernel_launches = launches;
    S.fit_terms = tab.n_q;
    S.n_capped_leaves = n_capped;
    S.n_device_allocs = plan->n_allocs;
    if (plan->timing) {
        float ms;
        // stage 7: the residual kernel alone (on the side stream when it overlaps the far
        // field); stage 8: the expansion kernel alone
        const int map[9][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 5}, {5, 6}, {6, 7}, {0, 7}, {8, 9}, {10, 7}};
        for (int i = 0; i < 9; ++i) {
            ms = 0;
            if (i < 7 || fast_leaf) cudaEventElapsedTime(&ms, plan->ev[map[i][0]], plan->ev[map[i][1]]);
            S.stage_ms[i] = ms;
        }
    }
    return DMK_OK;
}

dmk_status_t make_plan(int k, int D, const double L[3], double tol, int prec, int n_s, void* stream, dmk_plan_t* out) {
    if (!out) { g_plan_error = "out pointer is NULL"; return DMK_ERR_INVALID_ARG; }
    *out = nullptr;
    if (prec != DMK_FP64 && prec != DMK_MIXED) { g_plan_error = "precision must be DMK_FP64 or DMK_MIXED"; return DMK_ERR_INVALID_ARG; }
    if (n_s < 1) { g_plan_error = "n_s must be >= 1"; return DMK_ERR_INVALID_ARG; }
    dmk_plan_s* plan = new (std::nothrow) dmk_plan_s();
    if (!plan) { g_plan_error = "host allocation failed"; return DMK_ERR_OOM; }
    std::string err;
    dmk_status_t s = build_plan_tables(k, D, L, tol, plan->T, err);
    if (s != DMK_OK) { g_plan_error = err; delete plan; return s; }
    plan->prec = prec;
    plan->n_s = n_s;
    plan->stream = (cudaStream_t)stream;
    for (int i = 0; i < 3; ++i) {
        plan->geo.L[i] = plan->T.L[i];
        plan->geo.M[i] = plan->T.M[i];
        plan->geo.periodic[i] = plan->T.periodic[i];
    }
    plan->geo.s = plan->T.s;
    plan->geo.D = D;
    // exact reciprocals of powers of two (frexp mantissa 1/2); 0 marks "divide"
    auto inv_pow2 = [](double v) {
        int ex = 0;
        return std::frexp(v, &ex) == 0.5 ? 1.0 / v : 0.0;
    };
    plan->geo.inv_s_pow2 = inv_pow2(plan->T.s);
    for (int i = 0; i < 3; ++i) plan->geo.inv_L_pow2[i] = inv_pow2(plan->T.L[i]);
    for (int i = 0; i < 3; ++i) {
        plan->geo.wrap[i] = plan->T.wrap[i];
        plan->geo.origin[i] = plan->T.origin[i];
        plan->geo.padded[i] = plan->T.padded[i];
    }
    cudaError_t e = cudaGetDevice(&plan->device);
    if (e != cudaSuccess) { g_plan_error = std::string("no CUDA device: ") + cudaGetErrorString(e); delete plan; return DMK_ERR_CUDA; }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device);
    plan->smem_optin = (size_t)optin;
    cudaDeviceGetAttribute(&plan->n_sm, cudaDevAttrMultiProcessorCount, plan->device);
    if ((s = upload_tab<double>(plan, &plan->d_tab64, plan->tab64, 1e-17)) != DMK_OK ||
        (s = upload_tab<float>(plan, &plan->d_tab32, plan->tab32, 1e-9)) != DMK_OK || (s = upload_root(plan)) != DMK_OK) {
        g_plan_error = plan->err;
        dmk_destroy(plan);
        return s;
    }
    if (plan->T.padded[0] || plan->T.padded[1] || plan->T.padded[2]) {
        std::vector<int> cv(plan->T.cube_class);
        std::vector<int> cut;
        for (size_t m = 0; m < cv.size(); ++m)
            if (cv[m] == 1) cut.push_back((int)m);
        cv.push_back((int)cut.size());
        cv.insert(cv.end(), cut.begin(), cut.end());
        e = cudaMalloc((void**)&plan->d_cube, cv.size() * sizeof(int));
        if (e != cudaSuccess) { g_plan_error = "cube table allocation failed"; dmk_destroy(plan); return DMK_ERR_OOM; }
        ++plan->n_allocs;
        if (cudaMemcpy(plan->d_cube, cv.data(), cv.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
            g_plan_error = "cube table upload failed";
            dmk_destroy(plan);
            return DMK_ERR_CUDA;
        }
    }
    e = cudaMallocHost((void**)&plan->h_meta, 4096);
    if (e != cudaSuccess) {
        plan->h_meta = nullptr;
        g_plan_error = std::string("pinned host allocation failed: ") + cudaGetErrorString(e);
        dmk_destroy(plan);
        return DMK_ERR_OOM;
    }
    for (int i = 0; i < 11; ++i) cudaEventCreate(&plan->ev[i]);
    if (cudaStreamCreateWithFlags(&plan->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_cnt, cudaEventDisableTiming) != cudaSuccess) {
        g_plan_error = "stream or event creation failed";
        dmk_destroy(plan);
        return DMK_ERR_CUDA;
    }
    if (const char* v = std::getenv("DMK_PAIR_OVERLAP")) plan->pair_overlap = std::atoi(v) != 0;
    if (const char* v = std::getenv("DMK_PAIR_BLOCKS")) plan->pair_blocks = std::max(0, std::atoi(v));
    *out = plan;
    return DMK_OK;
}

}  // namespace

extern "C" {

dmk_status_t dmk_plan(dmk_kernel_t k, int D, double L1, double L2, double L3, double tol, dmk_plan_t* out) {
    const double L[3] = {L1, L2, L3};
    return make_plan(k, D, L, tol, DMK_MIXED, 250, nullptr, out);
}

dmk_status_t dmk_plan_ex(dmk_kernel_t k, int D, const double L[3], double tol, dmk_precision_t prec, int n_s,
                         void* cuda_stream, dmk_plan_t* out) {
    if (!L) { g_plan_error = "L is NULL"; return DMK_ERR_INVALID_ARG; }
    return make_plan(k, D, L, tol, prec, n_s, cuda_stream, out);
}

dmk_status_t dmk_eval(dmk_plan_t plan, int64_t N, const double* points, const double* strengths, double* potentials,
                      double* grad) {
    if (!plan) return DMK_ERR_INVALID_ARG;
    plan->err.clear();
    if (N < 0) { plan->err = "N < 0"; return DMK_ERR_INVALID_ARG; }
    if (N == 0) return DMK_OK;
    if (N > (int64_t)1 << 30) { plan->err = "N above 2^30"; return DMK_ERR_INVALID_ARG; }
    if (!points || !strengths || !potentials) { plan->err = "NULL array"; return DMK_ERR_INVALID_ARG; }
    cudaSetDevice(plan->device);
    if (plan->prec == DMK_FP64) return run_eval<double>(plan, plan->tab64, N, points, strengths, potentials, grad);
    return run_eval<float>(plan, plan->tab32, N, points, strengths, potentials, grad);
}

dmk_status_t dmk_eval_shard(dmk_plan_t plan, int64_t N, int64_t n_own, const double* points, const double* strengths,
                            double* potentials, double* grad, const int* cube_owned, dmk_chi_reduce_fn reduce,
                            void* ctx) {
    if (!plan) return DMK_ERR_INVALID_ARG;
    plan->err.clear();
    if (N < 0 || n_own < 0 || n_own > N) { plan->err = "need 0 <= n_own <= N"; return DMK_ERR_INVALID_ARG; }
    if (N > (int64_t)1 << 30) { plan->err = "N above 2^30"; return DMK_ERR_INVALID_ARG; }
    if (!cube_owned || !reduce) { plan->err = "cube_owned and reduce are required"; return DMK_ERR_INVALID_ARG; }
    if (plan->geo.padded[0] || plan->geo.padded[1] || plan->geo.padded[2]) {
        plan->err = "dmk_eval_shard: exact tilings only";
        return DMK_ERR_UNSUPPORTED;
    }
    if (N > 0 && (!points || !strengths || (n_own > 0 && !potentials))) { plan->err = "NULL array"; return DMK_ERR_INVALID_ARG; }
    cudaSetDevice(plan->device);
    EvalOpts sh{n_own, n_own, cube_owned, reduce, ctx};
    if (N == 0) {
        // nothing local, but the other ranks' reduction still needs this rank's (zero) share
        const RootTab& rt = plan->root;
        const int Mtot = plan->geo.M[0] * plan->geo.M[1] * plan->geo.M[2];
        const int64_t n = (int64_t)2 * (plan->T.root_dft ? 1 : Mtot) * plan->T.d_rho * (rt.nmode + plan->root2.nmode);
        void* vchi;
        CKS(ensure(plan, B_CHI, (size_t)(n + 2 * plan->T.d_rho) * sizeof(double), &vchi));
        CK(cudaMemsetAsync(vchi, 0, (size_t)(n + 2 * plan->T.d_rho) * sizeof(double), plan->stream));
        CKS(reduce_chi(plan, &sh, (Cx<double>*)vchi, n, (double*)vchi + n));
        CK(cudaStreamSynchronize(plan->stream));
        return DMK_OK;
    }
    if (plan->prec == DMK_FP64)
        return run_eval<double>(plan, plan->tab64, N, points, strengths, potentials, grad, &sh);
    return run_eval<float>(plan, plan->tab32, N, points, strengths, potentials, grad, &sh);
}

dmk_status_t dmk_eval_targets(dmk_plan_t plan, int64_t N, const double* sources, const double* strengths,
                              int64_t M, const double* targets, double* potentials, double* grad) {
    if (!plan) return DMK_ERR_INVALID_ARG;
    plan->err.clear();
    if (N < 0 || M < 0) { plan->err = "N < 0 or M < 0"; return DMK_ERR_INVALID_ARG; }
    if (M == 0) return DMK_OK;
    if (N + M > (int64_t)1 << 30) { plan->err = "N + M above 2^30"; return DMK_ERR_INVALID_ARG; }
    if ((N > 0 && (!sources || !strengths)) || !targets || !potentials) {
        plan->err = "NULL array";
        return DMK_ERR_INVALID_ARG;
    }
    cudaSetDevice(plan->device);
    // the targets enter the forest as points of zero strength, ahead of the sources: the tree
    // is built on both sets, the targets add nothing to any sum, and the self term of a target
    // (its own strength) vanishes
    const int drho = plan->T.d_rho;
    const int64_t Nt = M + N;
    void *vp, *vr;
    CKS(ensure(plan, B_TPTS, (size_t)Nt * 3 * sizeof(double), &vp));
    CKS(ensure(plan, B_TRHO, (size_t)Nt * drho * sizeof(double), &vr));
    double* pts = (double*)vp;
    double* rho = (double*)vr;
    const cudaStream_t st = plan->stream;
    CK(cudaMemcpyAsync(pts, targets, (size_t)M * 3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(rho, 0, (size_t)M * drho * sizeof(double), st));
    if (N > 0) {
        CK(cudaMemcpyAsync(pts + M * 3, sources, (size_t)N * 3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(rho + M * drho, strengths, (size_t)N * drho * sizeof(double), cudaMemcpyDeviceToDevice,
                           st));
    }
    EvalOpts opt{M, Nt, nullptr, nullptr, nullptr};
    if (plan->prec == DMK_FP64) return run_eval<double>(plan, plan->tab64, Nt, pts, rho, potentials, grad, &opt);
    return run_eval<float>(plan, plan->tab32, Nt, pts, rho, potentials, grad, &opt);
}

dmk_status_t dmk_eval_static(dmk_plan_t plan, int64_t N, const double* points, const double* strengths,
                             double* potentials, double* grad) {
    if (!plan) return DMK_ERR_INVALID_ARG;
    plan->err.clear();
    if (N < 0 || N > kStaticMaxN) {
        plan->err = "dmk_eval_static: N must lie in [0, " + std::to_string(kStaticMaxN) + "]";
        return DMK_ERR_INVALID_ARG;
    }
    if (N == 0) return DMK_OK;
    if (!points || !strengths || !potentials) { plan->err = "NULL array"; return DMK_ERR_INVALID_ARG; }
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) { plan->err = cudaGetErrorString(e); return DMK_ERR_CUDA; }
    if (plan->device < 0 || plan->device >= kMaxDevices) { plan->err = "device index out of range"; return DMK_ERR_CUDA; }
    void* base = nullptr;
    {
        // once per device, with that device current: the device address of the static array
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[plan->device]) {
            e = cudaGetSymbolAddress(&g_static_ptr[plan->device], g_static_workspace);
            if (e != cudaSuccess) {
                g_static_ptr[plan->device] = nullptr;
                plan->err = std::string("cudaGetSymbolAddress of the static workspace: ") + cudaGetErrorString(e);
                return DMK_ERR_CUDA;
            }
        }
        base = g_static_ptr[plan->device];
    }
    std::vector<DevBuf> saved;
    saved.swap(plan->bufs);            // the plan's own buffers are neither used nor freed
    plan->arena = (unsigned char*)base;
    plan->arena_cap = kStaticWorkspaceBytes;
    plan->arena_off = 0;
    dmk_status_t s = (plan->prec == DMK_FP64)
                         ? run_eval<double>(plan, plan->tab64, N, points, strengths, potentials, grad)
                         : run_eval<float>(plan, plan->tab32, N, points, strengths, potentials, grad);
    plan->arena = nullptr;
    plan->arena_cap = plan->arena_off = 0;
    plan->bufs.swap(saved);
    return s;
}

dmk_status_t dmk_vjp(dmk_plan_t plan, int64_t N, const double* points, const double* strengths,
                     const double* grad_u, const double* g, double* d_strengths, double* d_points) {
    if (!plan) return DMK_ERR_INVALID_ARG;
    plan->err.clear();
    if (N < 0) { plan->err = "N < 0"; return DMK_ERR_INVALID_ARG; }
    if (N == 0) return DMK_OK;
    if (N > (int64_t)1 << 30) { plan->err = "N above 2^30"; return DMK_ERR_INVALID_ARG; }
    if (!points || !strengths || !g || (d_points && !grad_u)) { plan->err = "NULL array"; return DMK_ERR_INVALID_ARG; }
    if (!d_strengths && !d_points) return DMK_OK;
    cudaSetDevice(plan->device);
    const int du = plan->T.d_u;
    if (plan->T.kernel == DMK_STRESSLET) {
        // three evaluations with the strengths g (x) e_m (k_vjp_stresslet_q)
        void *vq, *vu, *vgm;
        CKS(ensure(plan, B_VJPQ, (size_t)N * 9 * sizeof(double), &vq));
        CKS(ensure(plan, B_VJPV, (size_t)N * 3 * sizeof(double), &vu));
        if (d_points) CKS(ensure(plan, B_VJPG, (size_t)N * 9 * sizeof(double), &vgm));
        const cudaStream_t st = plan->stream;
        if (d_points)
            k_vjp_target<<<nblk(3 * N, 256), 256, 0, st>>>(N, 3, grad_u, g, d_points);
        for (int m = 0; m < 3; ++m) {
            k_vjp_stresslet_q<<<nblk(9 * N, 256), 256, 0, st>>>(N, m, g, (double*)vq);
            const dmk_status_t s = (plan->prec == DMK_FP64)
                ? run_eval<double>(plan, plan->tab64, N, points, (const double*)vq, (double*)vu,
                                   d_points ? (double*)vgm : nullptr)
                : run_eval<float>(plan, plan->tab32, N, points, (const double*)vq, (double*)vu,
                                  d_points ? (double*)vgm : nullptr);
            if (s != DMK_OK) return s;
            k_vjp_stresslet_acc<<<nblk(N, 256), 256, 0, st>>>(N, m, (const double*)vu, (const double*)vgm, strengths,
                                                              d_strengths, d_points);
        }
        CK(cudaGetLastError());
        CKS(host_wait(plan, st));
        return DMK_OK;
    }
    void *vv = d_strengths, *vg = nullptr;
    if (!vv) CKS(ensure(plan, B_VJPV, (size_t)N * du * sizeof(double), &vv));
    if (d_points) CKS(ensure(plan, B_VJPG, (size_t)N * 3 * du * sizeof(double), &vg));
    plan->allow_charged = 1;
    const dmk_status_t s = (plan->prec == DMK_FP64)
                               ? run_eval<double>(plan, plan->tab64, N, points, g, (double*)vv, (double*)vg)
                               : run_eval<float>(plan, plan->tab32, N, points, g, (double*)vv, (double*)vg);
    plan->allow_charged = 0;
    if (s != DMK_OK) return s;
    if (d_points) {
        k_vjp_points<<<nblk(3 * N, 256), 256, 0, plan->stream>>>(N, du, grad_u, g, (const double*)vg, strengths,
                                                                d_points);
        CK(cudaGetLastError());
        CKS(host_wait(plan, plan->stream));
    }
    return DMK_OK;
}

dmk_status_t dmk_eval_host(dmk_plan_t plan, int64_t N, const double* points, const double* strengths,
                           double* potentials, double* grad) {
    if (!plan) return DMK_ERR_INVALID_ARG;
    if (N == 0) return DMK_OK;
    if (N < 0 || !points || !strengths || !potentials) { plan->err = "bad arguments"; return DMK_ERR_INVALID_ARG; }
    const int drho = plan->T.d_rho, du = plan->T.d_u;
    void *dp, *dr, *du_, *dg = nullptr;
    dmk_status_t s;
    if ((s = ensure(plan, B_DEVPTS, 3 * N * sizeof(double), &dp)) != DMK_OK) return s;
    if ((s = ensure(plan, B_DEVRHO, N * drho * sizeof(double), &dr)) != DMK_OK) return s;
    if ((s = ensure(plan, B_DEVPOT, N * du * sizeof(double), &du_)) != DMK_OK) return s;
    if (grad && (s = ensure(plan, B_DEVGRAD, N * 3 * du * sizeof(double), &dg)) != DMK_OK) return s;
    cudaStream_t st = plan->stream;
    CK(cudaMemcpyAsync(dp, points, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dr, strengths, N * drho * sizeof(double), cudaMemcpyHostToDevice, st));
    s = dmk_eval(plan, N, (const double*)dp, (const double*)dr, (double*)du_, (double*)dg);
    if (s != DMK_OK) return s;
    CK(cudaMemcpyAsync(potentials, du_, N * du * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad) CK(cudaMemcpyAsync(grad, dg, N * 3 * du * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return DMK_OK;
}

dmk_status_t dmk_get_stats(dmk_plan_t plan, dmk_stats_t* out) {
    if (!plan || !out) return DMK_ERR_INVALID_ARG;
    *out = plan->stats;
    out->n_device_allocs = plan->n_allocs;
    return DMK_OK;
}

dmk_status_t dmk_set_pair_overlap(dmk_plan_t plan, int enable, int max_blocks_per_sm) {
    if (!plan || max_blocks_per_sm < 0) return DMK_ERR_INVALID_ARG;
    plan->pair_overlap = enable ? 1 : 0;
    plan->pair_blocks = max_blocks_per_sm;
    return DMK_OK;
}

dmk_status_t dmk_set_timing(dmk_plan_t plan, int enable) {
    if (!plan) return DMK_ERR_INVALID_ARG;
    plan->timing = enable ? 1 : 0;
    return DMK_OK;
}

dmk_status_t dmk_destroy(dmk_plan_t plan) {
    if (!plan) return DMK_OK;
    for (auto& b : plan->bufs)
        if (b.p) cudaFree(b.p);
    if (plan->d_tab64) cudaFree(plan->d_tab64);
    if (plan->d_tab32) cudaFree(plan->d_tab32);
    if (plan->d_root) cudaFree(plan->d_root);
    if (plan->d_root2) cudaFree(plan->d_root2);
    if (plan->d_self) cudaFree(plan->d_self);
    if (plan->d_cube) cudaFree(plan->d_cube);
    if (plan->side) {
        cudaStreamSynchronize(plan->side);
        cudaStreamDestroy(plan->side);
    }
    if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
    if (plan->ev_join) cudaEventDestroy(plan->ev_join);
    if (plan->ev_cnt) cudaEventDestroy(plan->ev_cnt);
    for (int i = 0; i < 11; ++i)
        if (plan->ev[i]) cudaEventDestroy(plan->ev[i]);
    if (plan->h_meta) cudaFreeHost(plan->h_meta);
    if (plan->h_chi) cudaFreeHost(plan->h_chi);
    delete plan;
    return DMK_OK;
}

dmk_status_t dmk_plan_info(dmk_kernel_t k, int D, const double L[3], double tol, dmk_plan_info_t* out) {
    if (!L || !out) { g_plan_error = "NULL argument"; return DMK_ERR_INVALID_ARG; }
    PlanTables T;
    std::string err;
    dmk_status_t s = build_plan_tables(k, D, L, tol, T, err);
    if (s != DMK_OK) { g_plan_error = err; return s; }
    auto nterms = [](const std::vector<double>& a, double tol_rel) {
        double mx = 0;
        for (double v : a) mx = std::max(mx, std::fabs(v));
        int n = (int)a.size();
        while (n > 1 && std::fabs(a[n - 1]) < tol_rel * mx) --n;
        return n;
    };
    out->c = T.c; out->s = T.s; out->R = T.R; out->dk = T.dk;
    out->p = T.p; out->n_f = T.nf; out->n_root_modes = T.n_root_modes;
    out->fit_terms_fp64 = nterms(T.fit_q, 1e-17);
    out->fit_terms_fp32 = nterms(T.fit_q, 1e-9);
    for (int i = 0; i < 3; ++i) { out->M[i] = T.M[i]; out->n_axis[i] = (int)T.kax[i].size(); }
    out->d_rho = T.d_rho; out->d_u = T.d_u;
    for (int part = 0; part < 2; ++part)
        for (int a = 0; a < 3; ++a) out->root_dft_len[3 * part + a] = T.root_dft_Q[part][a];
    return DMK_OK;
}

dmk_status_t dmk_plan_table(dmk_kernel_t k, int D, const double L[3], double tol, int which, double* out,
                            int64_t cap, int64_t* n) {
    if (!L || !n) { g_plan_error = "NULL argument"; return DMK_ERR_INVALID_ARG; }
    PlanTables T;
    std::string err;
    dmk_status_t s = build_plan_tables(k, D, L, tol, T, err);
    if (s != DMK_OK) { g_plan_error = err; return s; }
    std::vector<double> v;
    if (which == 0) {
        for (int i = 0; i < 3; ++i) v.insert(v.end(), T.kax[i].begin(), T.kax[i].end());
    } else if (which == 1) {
        for (auto& z : T.Wroot) { v.push_back(z.real()); v.push_back(z.imag()); }
    } else if (which == 2) {
        v = T.gdiff;
    } else if (which == 3) {
        v = {T.phi0, T.d2phi0, T.d2phihat0};
        v.insert(v.end(), T.phihat_samples.begin(), T.phihat_samples.end());
    } else if (which == 4) {
        v = herm_tables(T);
    } else if (which == 5) {
        for (int i = 0; i < 3; ++i) v.insert(v.end(), T.kax2[i].begin(), T.kax2[i].end());
    } else if (which == 6) {
        for (auto& z : T.Wroot2) { v.push_back(z.real()); v.push_back(z.imag()); }
    } else {
        g_plan_error = "which must be 0..6";
        return DMK_ERR_INVALID_ARG;
    }
    *n = (int64_t)v.size();
    if (out) std::memcpy(out, v.data(), sizeof(double) * (size_t)std::min<int64_t>(cap, (int64_t)v.size()));
    return DMK_OK;
}

const char* dmk_status_string(dmk_status_t s) {
    switch (s) {
        case DMK_OK: return "ok";
        case DMK_ERR_INVALID_ARG: return "invalid argument";
        case DMK_ERR_OUT_OF_DOMAIN: return "point outside the domain";
        case DMK_ERR_NOT_NEUTRAL: return "non-neutral charges for D = 1, 2 Laplace";
        case DMK_ERR_UNSUPPORTED: return "unsupported configuration";
        case DMK_ERR_TREE_DEPTH: return "tree depth limit";
        case DMK_ERR_OOM: return "out of device memory";
        case DMK_ERR_CUDA: return "CUDA error";
        case DMK_ERR_TIMEOUT: return "timeout";
    }
    return "unknown status";
}

const char* dmk_last_error(dmk_plan_t plan) {
    if (!plan) return g_plan_error.c_str();
    return plan->err.c_str();
}

}  // extern "C"
