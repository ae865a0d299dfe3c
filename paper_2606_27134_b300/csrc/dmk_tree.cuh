// Forest of octrees on the GPU (Sec. 3.1.1 and Sec. 4.1): quantised keys, radix sort,
// level-by-level refinement, 2:1 balance, colleague tables and leaf direct lists.
#pragma once
#include "dmk_device.cuh"

namespace dmk {

constexpr uint64_t kInvalidKey = ~0ULL;
constexpr int kErrDomain = 1;
constexpr int kErrNonFinite = 2;
constexpr int kErrIndex = 4;

// Integer coordinate of a (wrapped) coordinate v on axis a: floor(((v - origin) / s) 2^18),
// clamped to the tiled axis, with explicitly rounded FP64 operations (the same sequence as the
// oracle's quantisation).
__device__ __forceinline__ int quantize_axis(const Geo& g, int a, double v) {
    const double scale = (double)(1u << kBits);
    const double d = __dsub_rn(v, g.origin[a]);
    const double q = g.inv_s_pow2 != 0.0 ? __dmul_rn(d, g.inv_s_pow2) : __ddiv_rn(d, g.s);
    const double t = floor(__dmul_rn(q, scale));
    long long gi = (long long)t;
    const long long hi = ((long long)g.M[a] << kBits) - 1;
    gi = gi < 0 ? 0 : (gi > hi ? hi : gi);
    return (int)gi;
}

// Wrap periodic coordinates, quantise, and form the 64-bit key (cube << 54 | Morton of the
// 18-bit in-cube coordinates):
//   periodic: w = x - L floor(x / L); w >= L -> w - L; w < 0 -> 0.   free: w = x in [0, L).
// w (SoA, stride ws) keeps the wrapped coordinate itself; the origin enters the key only.
__device__ __forceinline__ double wrap_coord(const Geo& g, int a, double x, int* err) {
    const double L = g.L[a];
    double v;
    if (!isfinite(x)) {
        if (err) atomicOr(err, kErrNonFinite);
        x = 0.0;
    }
    if (g.wrap[a]) {
        const double f = floor(g.inv_L_pow2[a] != 0.0 ? __dmul_rn(x, g.inv_L_pow2[a]) : __ddiv_rn(x, L));
        v = __dsub_rn(x, __dmul_rn(L, f));
        if (v >= L) v = __dsub_rn(v, L);
        if (v < 0.0) v = 0.0;
    } else {
        v = x;
        if (!(v >= 0.0 && v < L)) {
            if (err) atomicOr(err, kErrDomain);
            v = 0.0;
        }
    }
    return v;
}

__global__ void k_quantize(int64_t N, const double* __restrict__ pts, Geo g, double* __restrict__ w, int64_t ws,
                           uint64_t* __restrict__ keys, int* __restrict__ idx, int* __restrict__ err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int G[3];
    for (int a = 0; a < 3; ++a) {
        const double v = wrap_coord(g, a, pts[3 * i + a], err);
        w[a * ws + i] = v;
        G[a] = quantize_axis(g, a, v);
    }
    keys[i] = cell_key(g, kBits, G);
    idx[i] = (int)i;
}

// Periodic images of the sources along the padded axes (Sec. 4.1.2): every w + sum_i n_i L_i e_i
// (n_i in -3..3 over the padded axes, n = 0 excluded) inside Omega_ext = [origin, origin + M s).
// Image enumeration: n in lexicographic order over the padded axes, the lowest axis slowest.
__device__ __forceinline__ int image_combos(const Geo& g, int* axes) {
    int k = 0;
    for (int a = 0; a < 3; ++a)
        if (g.padded[a]) axes[k++] = a;
    return k;
}
__device__ __forceinline__ bool image_of(const Geo& g, const double v[3], int na, const int* axes, int combo,
                                         double out[3]) {
    int n[3] = {0, 0, 0};
    int c = combo;
    bool zero = true;
    for (int j = na - 1; j >= 0; --j) {
        n[j] = c % 7 - 3;
        c /= 7;
        zero = zero && n[j] == 0;
    }
    if (zero) return false;
    for (int a = 0; a < 3; ++a) out[a] = v[a];
    for (int j = 0; j < na; ++j) {
        const int a = axes[j];
        out[a] = __dadd_rn(v[a], __dmul_rn((double)n[j], g.L[a]));
        const double lo = g.origin[a], hi = __dadd_rn(g.origin[a], (double)g.M[a] * g.s);
        if (!(out[a] >= lo && out[a] < hi)) return false;
    }
    return true;
}

// images per point (cnt[i]); with FILL, the images after the N originals at off[i] in point
// order: wrapped coordinate, key, point index N + off[i] + j and its source src[...] = i
template <bool FILL>
__global__ void k_images(int64_t N, const double* __restrict__ pts, Geo g, double* __restrict__ w, int64_t ws,
                         int* __restrict__ cnt, const int* __restrict__ off, uint64_t* __restrict__ keys,
                         int* __restrict__ idx, int* __restrict__ src) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int axes[3];
    const int na = image_combos(g, axes);
    int ncombo = 1;
    for (int j = 0; j < na; ++j) ncombo *= 7;
    double v[3];
    if (FILL) {
        for (int a = 0; a < 3; ++a) v[a] = w[a * ws + i];
    } else {
        for (int a = 0; a < 3; ++a) v[a] = wrap_coord(g, a, pts[3 * i + a], nullptr);
    }
    int k = 0;
    for (int combo = 0; combo < ncombo; ++combo) {
        double im[3];
        if (!image_of(g, v, na, axes, combo, im)) continue;
        if (FILL) {
            const int64_t j = N + off[i] + k;
            int G[3];
            for (int a = 0; a < 3; ++a) {
                w[a * ws + j] = im[a];
                G[a] = quantize_axis(g, a, im[a]);
            }
            keys[j] = cell_key(g, kBits, G);
            idx[j] = (int)j;
            src[j] = (int)i;
        }
        ++k;
    }
    if (!FILL) cnt[i] = k;
    if (FILL && i < N) src[i] = (int)i;
}

// sorted order -> sorted SoA coordinates and strengths
// Gather into key order (FP64 coordinates and strengths; FP32 two-part copies for the mixed
// path) and per-block sums of the strengths and of their absolute values (block b writes
// partial[b * 2 d_rho + v], v < d_rho: sum rho_v, v >= d_rho: sum |rho_v|).
constexpr int kGatherThreads = 256;

// FP32 path: one record per sorted point, read whole by the leaf kernels (one 32-byte sector
// for d_rho = 1): floats 0-2 the leading FP32 parts of the coordinates, 4-6 the trailing
// parts (exact split of the FP64 value to 48 bits), the strengths in FP32 at 3, 7, 8, 9, ...
// Records of 8 floats for d_rho = 1, else 16.
__host__ __device__ constexpr int point_record_floats(int drho) { return drho <= 1 ? 8 : 16; }
__host__ __device__ constexpr int point_record_rho(int a) { return a == 0 ? 3 : (a == 1 ? 7 : 6 + a); }

// N points (originals and images), N0 originals; src maps a point to its original (NULL: the
// identity, no images).  Coordinates leave in the frame of Omega_ext's lower corner, x - origin;
// orig[k] = the original index of sorted point k.  The strength sums count the originals only.
__global__ void __launch_bounds__(kGatherThreads) k_gather(int64_t N, int64_t N0, int drho, const int* __restrict__ idx,
                                                           const int* __restrict__ src, Geo g,
                                                           const double* __restrict__ w,
                                                           const double* __restrict__ rho, double* __restrict__ xs,
                                                           double* __restrict__ rs, float* __restrict__ pk,
                                                           int* __restrict__ orig, double* __restrict__ partial) {
    __shared__ double red[18][kGatherThreads / 32];
    const int64_t k = blockIdx.x * (int64_t)kGatherThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s[9], sa[9];
    for (int a = 0; a < drho; ++a) { s[a] = 0; sa[a] = 0; }
    if (k < N) {
        const int i = idx[k];
        const int io = src ? src[i] : i;
        if (orig) orig[k] = io;
        float rec[16];
        const int nf = point_record_floats(drho);
        for (int f = 0; f < 16; ++f) rec[f] = 0.0f;
        for (int a = 0; a < 3; ++a) {
            const double v = __dsub_rn(w[a * N + i], g.origin[a]);
            xs[a * N + k] = v;
            const float h = (float)v;
            rec[a] = h;
            rec[4 + a] = (float)(v - (double)h);
        }
        for (int a = 0; a < drho; ++a) {
            const double r = rho[(int64_t)io * drho + a];
            rs[k * drho + a] = r;
            rec[point_record_rho(a)] = (float)r;
            if (i < N0) {
                s[a] = r;
                sa[a] = fabs(r);
            }
        }
        if (pk) {
            float4* dst = reinterpret_cast<float4*>(pk + k * nf);
            for (int f = 0; f < nf / 4; ++f) dst[f] = make_float4(rec[4 * f], rec[4 * f + 1], rec[4 * f + 2], rec[4 * f + 3]);
        }
    }
    for (int a = 0; a < drho; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            s[a] += __shfl_down_sync(0xffffffffu, s[a], o);
            sa[a] += __shfl_down_sync(0xffffffffu, sa[a], o);
        }
        if (lane == 0) { red[a][warp] = s[a]; red[drho + a][warp] = sa[a]; }
    }
    __syncthreads();
    if (threadIdx.x < 2 * drho) {
        double t = 0;
        for (int q = 0; q < kGatherThreads / 32; ++q) t += red[threadIdx.x][q];
        partial[(size_t)blockIdx.x * 2 * drho + threadIdx.x] = t;
    }
}

// one CTA: out[v] = sum over blocks of partial[b * nv + v], in a fixed order (warp per value)
__global__ void k_sum_partials(int nb, int nv, const double* __restrict__ partial, double* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int v = warp; v < nv; v += nwarp) {
        double t = 0;
        for (int b = lane; b < nb; b += 32) t += partial[(size_t)b * nv + v];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) out[v] = t;
    }
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* a, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int64_t upper_bound_u64(const uint64_t* a, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
// exact-match search; -1 if absent
__device__ __forceinline__ int64_t find_u64(const uint64_t* a, int64_t n, uint64_t v) {
    int64_t i = lower_bound_u64(a, n, v);
    return (i < n && a[i] == v) ? i : -1;
}

// point range of a cell at `level` in the sorted point keys
__device__ __forceinline__ void cell_range(const uint64_t* pkeys, int64_t N, int level, uint64_t key,
                                           int64_t& lo, int64_t& hi) {
    int sh = 3 * (kBits - level);
    uint64_t first = key << sh;
    uint64_t last = first | ((sh == 0) ? 0ULL : ((1ULL << sh) - 1ULL));
    lo = lower_bound_u64(pkeys, N, first);
    hi = upper_bound_u64(pkeys, N, last);
}

// ---- refinement (Sec. 3.1.1), one pass over the sorted points --------------------------------
// The cells of level l are the runs of equal key >> 3(kBits - l) in the sorted point keys.  A
// cell splits iff it holds more than n_s points (and l < kBits), i.e. its run, starting at i,
// still covers i + n_s.  A split cell's parent holds at least as many points and splits too, so
// the split cells of every level follow from one pass over the points; they come out in key
// order through an order-preserving compaction: per-block counts, a one-CTA scan, a write pass.
// Only levels l < lmax are examined: the keys may be sorted on their leading 3 lmax bits only
// (plus the cube index), which orders every cell of those levels.
constexpr int kRefineThreads = 256;

struct SplitProbe {
    uint64_t k0, km1, kns;
    bool first, has_ns;
    __device__ __forceinline__ SplitProbe(const uint64_t* pk, int64_t N, int64_t i, int n_s) {
        first = (i == 0);
        has_ns = i + n_s < N;
        k0 = pk[i];
        km1 = first ? 0 : pk[i - 1];
        kns = has_ns ? pk[i + n_s] : 0;
    }
    // point i starts a level-l cell with more than n_s points
    __device__ __forceinline__ bool split(int l) const {
        const int sh = 3 * (kBits - l);
        const uint64_t c = k0 >> sh;
        return (first || (km1 >> sh) != c) && has_ns && (kns >> sh) == c;
    }
};

// counts of split-cell starts per level and block: bcnt[l * nblk + block].  With the keys sorted
// on all their bits (lmax = kBits), also counts into *capped the cells at the depth cap (level
// kBits, never split) that hold more than n_s points: they stay leaves.
__global__ void __launch_bounds__(kRefineThreads) k_refine_count(int64_t N, const uint64_t* __restrict__ pk, int n_s,
                                                                 int nblk, int lmax, int* __restrict__ bcnt,
                                                                 int* __restrict__ capped) {
    __shared__ int wc[kBits][kRefineThreads / 32];
    const int64_t i = blockIdx.x * (int64_t)kRefineThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool valid = i < N;
    SplitProbe sp(pk, N, valid ? i : 0, n_s);
    for (int l = 0; l < kBits; ++l) {
        const unsigned bal = __ballot_sync(0xffffffffu, valid && l < lmax && sp.split(l));
        if (lane == 0) wc[l][warp] = __popc(bal);
    }
    const unsigned cap_bal = __ballot_sync(0xffffffffu, valid && lmax >= kBits && sp.split(kBits));
    if (lane == 0 && cap_bal) atomicAdd(capped, __popc(cap_bal));
    __syncthreads();
    if (threadIdx.x < kBits) {
        int sum = 0;
        for (int w = 0; w < kRefineThreads / 32; ++w) sum += wc[threadIdx.x][w];
        bcnt[threadIdx.x * nblk + blockIdx.x] = sum;
    }
}

// one CTA: exclusive scan of the block counts of every level -> boff, totals -> nR[l].  A level
// with no split cell has none below it, so the scan stops at the first empty level.
__global__ void __launch_bounds__(1024) k_refine_scan(int nblk, const int* __restrict__ bcnt, int* __restrict__ boff,
                                                      int* __restrict__ nR) {
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (nblk + 1023) / 1024;
    const int b0 = min(nblk, t * per), b1 = min(nblk, b0 + per);
    int done = 0;
    for (int l = 0; l < kBits; ++l) {
        const int* c = bcnt + (size_t)l * nblk;
        int s = 0;
        for (int b = b0; b < b1; ++b) s += c[b];
        int x = s;                                     // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int v = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        int run = x - s + (w > 0 ? wsum[w - 1] : 0);
        for (int b = b0; b < b1; ++b) {
            boff[(size_t)l * nblk + b] = run;
            run += c[b];
        }
        const int total = wsum[31];
        if (t == 0) nR[l] = total;
        done = l + 1;
        __syncthreads();
        if (total == 0) break;
    }
    if (t == 0)
        for (int l = done; l <= kBits; ++l) nR[l] = 0;   // level kBits never splits
}

// split cells of level l, in key order: R[l * cap + k]
__global__ void __launch_bounds__(kRefineThreads) k_refine_write(int64_t N, const uint64_t* __restrict__ pk, int n_s,
                                                                 int nblk, int lmax, const int* __restrict__ boff,
                                                                 int64_t cap, uint64_t* __restrict__ R) {
    __shared__ int wc[kBits][kRefineThreads / 32];
    const int64_t i = blockIdx.x * (int64_t)kRefineThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool valid = i < N;
    SplitProbe sp(pk, N, valid ? i : 0, n_s);
    unsigned bals[kBits];
    for (int l = 0; l < kBits; ++l) {
        bals[l] = __ballot_sync(0xffffffffu, valid && l < lmax && sp.split(l));
        if (lane == 0) wc[l][warp] = __popc(bals[l]);
    }
    __syncthreads();
    if (threadIdx.x < kBits) {                         // exclusive prefix over the warps
        int run = 0;
        for (int w = 0; w < kRefineThreads / 32; ++w) {
            const int v = wc[threadIdx.x][w];
            wc[threadIdx.x][w] = run;
            run += v;
        }
    }
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    for (int l = 0; l < kBits; ++l) {
        if (bals[l] & (1u << lane)) {
            const int pos = boff[(size_t)l * nblk + blockIdx.x] + wc[l][warp] + __popc(bals[l] & below);
            R[(size_t)l * cap + pos] = sp.k0 >> (3 * (kBits - l));
        }
    }
}

// Balance check of every level at once: counts, per level l - 1, the parents of neighbours of
// level-l non-leaf cells that are not non-leaf (missing[l - 1]).  All zero means the refined
// forest is already 2:1 balanced.
__global__ void k_balance_check(int64_t cap, const uint64_t* __restrict__ R, const int* __restrict__ nR, Geo g,
                                int* __restrict__ missing) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per = 27 * cap;
    if (t >= (int64_t)(kBits - 1) * per) return;
    const int l = 1 + (int)(t / per);
    const int64_t r = t % per;
    const int i = (int)(r / 27), d = (int)(r % 27);
    if (i >= nR[l]) return;
    const int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    int ix[3], nb[3], sh[3];
    cell_ix(g, l, R[(size_t)l * cap + i], ix);
    if (!neighbour(g, l, ix, dd, nb, sh)) return;
    const int par[3] = {nb[0] >> 1, nb[1] >> 1, nb[2] >> 1};
    if (find_u64(R + (size_t)(l - 1) * cap, nR[l - 1], cell_key(g, l - 1, par)) < 0) atomicAdd(&missing[l - 1], 1);
}

// 2:1 balance, bottom-up: every non-leaf cell at level l needs all its neighbour cells at
// level l to exist, i.e. their parents (level l-1) must be non-leaf.  Writes the parents of
// the 27 neighbours of the first nR[0] cells of R (a neighbour outside a free axis stands in
// its own cell's parent, already required), then the current non-leaf cells of level l-1,
// then kInvalidKey padding up to 27 capR + capP entries.
__global__ void k_balance_cand(int capR, const uint64_t* __restrict__ R, const int* __restrict__ nR, int capP,
                               const uint64_t* __restrict__ Rp, const int* __restrict__ nRp, int level, Geo g,
                               uint64_t* __restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 27 * capR + capP) return;
    if (t < 27 * capR) {
        const int i = t / 27, d = t % 27;
        if (i >= nR[0]) { out[t] = kInvalidKey; return; }
        int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
        int ix[3], nb[3], sh[3];
        cell_ix(g, level, R[i], ix);
        if (!neighbour(g, level, ix, dd, nb, sh))
            for (int a = 0; a < 3; ++a) nb[a] = ix[a];
        int par[3] = {nb[0] >> 1, nb[1] >> 1, nb[2] >> 1};
        out[t] = cell_key(g, level - 1, par);
    } else {
        const int j = t - 27 * capR;
        out[t] = (j < nRp[0]) ? Rp[j] : kInvalidKey;
    }
}

// 2:1 balance of one level in one CTA, for levels with few non-leaf cells: the parents of the
// neighbours of the non-leaf cells of level l that are not yet non-leaf at level l - 1 are
// collected, deduplicated and ordered by rank, and merged with R_{l-1} into Rout (sorted), with
// the new count in nR[l - 1].  More than kBalNew such cells sets *overflow and leaves nR
// unchanged; the caller then balances with the general path.  A set *overflow also makes later
// levels return at once.
constexpr int kBalThreads = 1024;
constexpr int kBalNew = 1024;
constexpr int kBalCache = 2048;     // R_{l-1} searched in shared memory up to this size

__global__ void __launch_bounds__(kBalThreads) k_balance_small(const uint64_t* __restrict__ R,
                                                               const uint64_t* __restrict__ Rp, int* __restrict__ nR,
                                                               int l, Geo g, uint64_t* __restrict__ Rout,
                                                               int* __restrict__ overflow) {
    __shared__ uint64_t nw[kBalNew];
    __shared__ uint64_t U[kBalNew];
    __shared__ uint64_t Rc[kBalCache];
    __shared__ unsigned char fst[kBalNew];
    __shared__ int cnt, nu;
    if (*overflow) return;
    const int n = nR[l], m = nR[l - 1];
    if (threadIdx.x == 0) { cnt = 0; nu = 0; }
    if (m <= kBalCache)
        for (int a = threadIdx.x; a < m; a += blockDim.x) Rc[a] = Rp[a];
    const uint64_t* Rs = (m <= kBalCache) ? Rc : Rp;
    __syncthreads();
    for (int t = threadIdx.x; t < 27 * n; t += blockDim.x) {
        const int i = t / 27, d = t % 27;
        const int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
        int ix[3], nb[3], sh[3];
        cell_ix(g, l, R[i], ix);
        if (!neighbour(g, l, ix, dd, nb, sh)) continue;
        const int par[3] = {nb[0] >> 1, nb[1] >> 1, nb[2] >> 1};
        const uint64_t P = cell_key(g, l - 1, par);
        if (find_u64(Rs, m, P) < 0) {
            const int k = atomicAdd(&cnt, 1);
            if (k < kBalNew) nw[k] = P;
        }
    }
    __syncthreads();
    const int k = cnt;
    if (k > kBalNew) {
        if (threadIdx.x == 0) *overflow = 1;
        return;
    }
    // distinct new cells in key order: the first occurrence of each value goes to its rank among
    // the distinct values
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
        const uint64_t v = nw[a];
        bool first = true;
        for (int b = 0; b < a && first; ++b) first = nw[b] != v;
        fst[a] = first ? 1 : 0;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
        if (!fst[a]) continue;
        const uint64_t v = nw[a];
        int r = 0;
        for (int b = 0; b < k; ++b) r += (fst[b] && nw[b] < v) ? 1 : 0;
        U[r] = v;
        atomicAdd(&nu, 1);
    }
    __syncthreads();
    const int u = nu;
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
        const uint64_t x = Rp[a];
        Rout[a + lower_bound_u64(U, u, x)] = x;
    }
    for (int b = threadIdx.x; b < u; b += blockDim.x) {
        const uint64_t y = U[b];
        Rout[b + lower_bound_u64(Rs, m, y)] = y;
    }
    if (threadIdx.x == 0) nR[l - 1] = m + u;
}

// after sort + unique the padding key (largest) may remain once at the end: drop it
__global__ void k_trim_invalid(const uint64_t* __restrict__ sorted_unique, int* __restrict__ count) {
    const int n = count[0];
    if (n > 0 && sorted_unique[n - 1] == kInvalidKey) count[0] = n - 1;
}


struct BoxArrays {
    uint64_t* key;   // cell key (level-local)
    int* level;
    int* ix;         // 3 per box
    int* start;      // sorted point range
    int* end;
    int* child0;     // first of 8 children, -1 for leaves
    int* parent;     // -1 for roots
    int* nl;         // index among non-leaf boxes, -1 for leaves
    int* coll;       // 27 per box: colleague box or -1
};

// per-level arrays of the forest, passed by value to the all-level kernels below.  The cells of
// level 0 are the cubes 0..Mtot-1; the cells of level l > 0 are the eight children of each
// non-leaf cell of level l - 1, in key order: cell i = R_{l-1}[i / 8] * 8 + i % 8.
struct LevelSet {
    const uint64_t* R[kMaxLevels + 1];       // sorted non-leaf cells of each level
    int off[kMaxLevels + 2];                 // first box of each level
    int nl_off[kMaxLevels + 2];              // first non-leaf index of each level
    int nR[kMaxLevels + 1];
    int nlev;
};

__device__ __forceinline__ int level_of(const int* off, int nlev, int b) {
    int l = 0;
    while (l + 1 < nlev && off[l + 1] <= b) ++l;
    return l;
}

__device__ __forceinline__ uint64_t level_cell(const LevelSet& ls, int l, int i) {
    return l == 0 ? (uint64_t)i : ((ls.R[l - 1][i >> 3] << 3) | (uint64_t)(i & 7));
}

// Boxes of every level in one launch: key, level, index, point range, first child, parent,
// non-leaf index (and the non-leaf list), and the leaf flags for the leaf compaction.
__global__ void k_box_fill_all(LevelSet ls, int nb, const uint64_t* __restrict__ pkeys, int64_t N, Geo g,
                               BoxArrays B, int* __restrict__ nl_box, int* __restrict__ leaf_flag,
                               int* __restrict__ iota) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int level = level_of(ls.off, ls.nlev, b);
    const int i = b - ls.off[level];
    const uint64_t key = level_cell(ls, level, i);
    B.key[b] = key;
    B.level[b] = level;
    int ix[3];
    cell_ix(g, level, key, ix);
    B.ix[3 * b] = ix[0];
    B.ix[3 * b + 1] = ix[1];
    B.ix[3 * b + 2] = ix[2];
    int64_t lo, hi;
    cell_range(pkeys, N, level, key, lo, hi);
    B.start[b] = (int)lo;
    B.end[b] = (int)hi;
    const int nRl = ls.nR[level];
    const int64_t r = (nRl > 0) ? find_u64(ls.R[level], nRl, key) : -1;
    B.child0[b] = (r >= 0) ? ls.off[level + 1] + 8 * (int)r : -1;
    if (r >= 0) {
        B.nl[b] = ls.nl_off[level] + (int)r;
        nl_box[ls.nl_off[level] + r] = b;
    } else {
        B.nl[b] = -1;
    }
    // parent: the level-(l-1) cell R_{l-1}[i / 8]; its box index there
    if (level == 0) {
        B.parent[b] = -1;
    } else {
        const int pl = level - 1;
        const uint64_t pkey = key >> 3;
        int64_t pi;
        if (pl == 0) {
            pi = (int64_t)pkey;
        } else {
            const int64_t gi = find_u64(ls.R[pl - 1], ls.nR[pl - 1], pkey >> 3);
            pi = (gi < 0) ? -1 : gi * 8 + (int64_t)(pkey & 7);
        }
        B.parent[b] = (pi >= 0) ? ls.off[pl] + (int)pi : -1;
    }
    leaf_flag[b] = (r < 0 && hi > lo) ? 1 : 0;
    iota[b] = b;
}

// colleague table: coll[b * 27 + d] = box at the same level with offset d, or -1
__global__ void k_colleagues(int nb, const int* __restrict__ level, const int* __restrict__ ixa,
                             const uint64_t* __restrict__ keys, LevelSet ls, Geo g, int* __restrict__ coll) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 27 * nb) return;
    int b = t / 27, d = t % 27;
    int l = level[b];
    int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    int ix[3] = {ixa[3 * b], ixa[3 * b + 1], ixa[3 * b + 2]};
    int nbx[3], sh[3];
    int res = -1;
    if (neighbour(g, l, ix, dd, nbx, sh)) {
        uint64_t k = cell_key(g, l, nbx);
        int64_t pos = find_u64(keys + ls.off[l], ls.off[l + 1] - ls.off[l], k);
        if (pos >= 0) res = ls.off[l] + (int)pos;
    }
    coll[t] = res;
}

// Direct list of target leaf T (telescoping recursion of the split, Eqs. multilevel_ks,
// u_four_partsDP, Sec. 3.1.5):
//   (a) for j < level(T): leaf colleagues C of T's level-j ancestor, kernel K_R(nu_j);
//   (b) every colleague C of T (leaf or not: all points below it), kernel K_R(nu_level(T)).
// Entry = {start, end, packed shifts and level, unused}.
struct DirectEntry { int start, end, code, pad; };

// Residual-sum tasks of the leaf stage: a tile of m consecutive targets of one leaf, m =
// kPairTile for the full tiles and one tile per set bit of nt mod kPairTile for the rest; as
// (leaf index, first target offset within the leaf, m, 0).  Consecutive targets are close in
// key order, so a tile is spatially compact.
constexpr int kPairTileLog = 4;
constexpr int kPairTile = 1 << kPairTileLog;

// task k of a leaf with nt targets: full tiles first, then the remainder's set bits high to low
__device__ __forceinline__ int4 pair_task(int li, int nt, int k) {
    const int a = nt >> kPairTileLog;
    if (k < a) return make_int4(li, kPairTile * k, kPairTile, 0);
    int rem = nt & (kPairTile - 1), t0 = kPairTile * a, j = k - a;
    while (true) {
        const int bit = 31 - __clz(rem);
        if (j == 0) return make_int4(li, t0, 1 << bit, 0);
        t0 += 1 << bit;
        rem &= ~(1 << bit);
        --j;
    }
}

// number of such tasks
__device__ __forceinline__ int pair_task_count(int nt) { return (nt >> kPairTileLog) + __popc(nt & (kPairTile - 1)); }


__device__ __forceinline__ int pack_code(const int sh[3], int level) {
    return (sh[0] + 1) | ((sh[1] + 1) << 2) | ((sh[2] + 1) << 4) | (level << 6);
}

// Per leaf: the direct-list entry count and the residual-task count (pair_task_count) at
// counts[i] and counts[tbase + i] (FILL = false); after one exclusive scan over both halves,
// the entries and the leaf's tasks (pair_task) at offs[i] and offs[tbase + i] - offs[tbase].
template <bool FILL>
__global__ void k_direct(int cap, const int* __restrict__ nleaf_dev, const int* __restrict__ leaves, BoxArrays B,
                         Geo g, int* __restrict__ counts, const int* __restrict__ offs, DirectEntry* __restrict__ out,
                         unsigned long long* __restrict__ npairs, int tbase, int4* __restrict__ tasks) {
    // one warp per leaf, lane d < 27 = colleague offset; entries in the order (ancestor level
    // descending, then the leaf's own colleagues), d ascending within a level
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= cap) return;
    if (i >= nleaf_dev[0]) {
        if (!FILL && lane == 0) counts[i] = counts[tbase + i] = 0;
        return;
    }
    const int T = leaves[i];
    const int lT = B.level[T];
    const int nt = B.end[T] - B.start[T];
    if (FILL) {
        const int t0 = offs[tbase + i] - offs[tbase], ntask = pair_task_count(nt);
        for (int k = lane; k < ntask; k += 32) tasks[t0 + k] = pair_task(i, nt, k);
    }
    const unsigned below = (1u << lane) - 1u;
    int pos = FILL ? offs[i] : 0;
    int cnt = 0;
    long long pairs = 0;
    auto visit = [&](int box, int j, bool need_leaf) {
        const int d = lane;
        int C = -1;
        if (d < 27) {
            C = B.coll[box * 27 + d];
            if (C >= 0 && ((need_leaf && B.child0[C] >= 0) || B.end[C] <= B.start[C])) C = -1;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, C >= 0);
        if (C >= 0) {
            if (FILL) {
                const int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
                const int ix[3] = {B.ix[3 * box], B.ix[3 * box + 1], B.ix[3 * box + 2]};
                int nbx[3], sh[3];
                neighbour(g, j, ix, dd, nbx, sh);
                out[pos + __popc(bal & below)] = {B.start[C], B.end[C], pack_code(sh, j), 0};
            } else {
                pairs += (long long)(B.end[C] - B.start[C]) * nt;
            }
        }
        pos += __popc(bal);
        cnt += __popc(bal);
    };
    int A = B.parent[T];
    for (int j = lT - 1; j >= 0; --j) {         // (a) leaf colleagues of the ancestors
        visit(A, j, true);
        A = B.parent[A];
    }
    visit(T, lT, false);                         // (b) every colleague of T
    if (!FILL) {
        for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        if (lane == 0) {
            counts[i] = cnt;
            counts[tbase + i] = pair_task_count(nt);
            atomicAdd(npairs, (unsigned long long)pairs);
        }
    }
}

}  // namespace dmk
