// Forest of octrees on the GPU (Sec. 3.1.1 and Sec. 4.1): quantised keys, radix sort,
// level-by-level refinement, 2:1 balance, colleague tables and leaf direct lists.
#pragma once
#include "dmk_device.cuh"

namespace dmk {

constexpr uint64_t kInvalidKey = ~0ULL;
constexpr int kErrDomain = 1;
constexpr int kErrNonFinite = 2;
constexpr int kErrIndex = 4;

// Wrap periodic coordinates, quantise, and form the 64-bit key (cube << 54 | Morton of the
// 18-bit in-cube coordinates).  The arithmetic uses explicitly rounded FP64 operations so
// that the integer coordinates are exactly floor((w / s) * 2^18):
//   periodic: w = x - L floor(x / L); w >= L -> w - L; w < 0 -> 0.   free: w = x in [0, L).
__global__ void k_quantize(int64_t N, const double* __restrict__ pts, Geo g, double* __restrict__ w,
                           uint64_t* __restrict__ keys, int* __restrict__ idx, int* __restrict__ err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int G[3];
    const double scale = (double)(1u << kBits);
    for (int a = 0; a < 3; ++a) {
        double x = pts[3 * i + a];
        double L = g.L[a];
        double v;
        if (!isfinite(x)) { atomicOr(err, kErrNonFinite); x = 0.0; }
        if (g.periodic[a]) {
            double f = floor(__ddiv_rn(x, L));
            v = __dsub_rn(x, __dmul_rn(L, f));
            if (v >= L) v = __dsub_rn(v, L);
            if (v < 0.0) v = 0.0;
        } else {
            v = x;
            if (!(v >= 0.0 && v < L)) { atomicOr(err, kErrDomain); v = 0.0; }
        }
        w[a * N + i] = v;
        double t = floor(__dmul_rn(__ddiv_rn(v, g.s), scale));
        long long gi = (long long)t;
        long long hi = ((long long)g.M[a] << kBits) - 1;
        gi = gi < 0 ? 0 : (gi > hi ? hi : gi);
        G[a] = (int)gi;
    }
    keys[i] = cell_key(g, kBits, G);
    idx[i] = (int)i;
}

// sorted order -> sorted SoA coordinates and strengths
__global__ void k_gather(int64_t N, int drho, const int* __restrict__ idx, const double* __restrict__ w,
                         const double* __restrict__ rho, double* __restrict__ xs, double* __restrict__ rs,
                         float* __restrict__ xh, float* __restrict__ xl, float* __restrict__ rsf) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N) return;
    int i = idx[k];
    for (int a = 0; a < 3; ++a) {
        const double v = w[a * N + i];
        xs[a * N + k] = v;
        if (xh) {   // leading + trailing FP32 parts (exact split of the FP64 value to 48 bits)
            const float h = (float)v;
            xh[a * N + k] = h;
            xl[a * N + k] = (float)(v - (double)h);
        }
    }
    for (int a = 0; a < drho; ++a) {
        const double r = rho[(int64_t)i * drho + a];
        rs[k * drho + a] = r;
        if (rsf) rsf[k * drho + a] = (float)r;
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

// Refinement and balance run on device-side counters: the host sizes every array by an upper
// bound and the kernels read the actual counts, so no host round trip is needed per level.

// refinement rule (Sec. 3.1.1): split iff the cell holds more than n_s points (and level < cap).
// Cells of `level`: ncell = ncell0 at level 0, else 8 * (non-leaf count of level - 1).
__global__ void k_split_flags(int cap, const uint64_t* __restrict__ cells, int level, int ncell0,
                              const int* __restrict__ nR_prev, const uint64_t* __restrict__ pkeys, int64_t N,
                              int n_s, int* __restrict__ flags) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    const int ncell = (level == 0) ? ncell0 : 8 * nR_prev[0];
    if (i >= ncell) { flags[i] = 0; return; }
    int64_t lo, hi;
    cell_range(pkeys, N, level, cells[i], lo, hi);
    flags[i] = (hi - lo > n_s && level < kBits) ? 1 : 0;
}

// children of the first nR[0] cells of R (8 each, in key order)
__global__ void k_children(int cap8, const uint64_t* __restrict__ R, const int* __restrict__ nR,
                           uint64_t* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap8 || (i >> 3) >= nR[0]) return;
    out[i] = (R[i >> 3] << 3) | (uint64_t)(i & 7);
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

// after sort + unique the padding key (largest) may remain once at the end: drop it
__global__ void k_trim_invalid(const uint64_t* __restrict__ sorted_unique, int* __restrict__ count) {
    const int n = count[0];
    if (n > 0 && sorted_unique[n - 1] == kInvalidKey) count[0] = n - 1;
}

// level-0 cells: every cube of the tiling, in key (= cube) order
__global__ void k_iota_u64(int n, uint64_t* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint64_t)i;
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

// fills the boxes of one level: cells_l sorted; R_l sorted non-leaf subset; parents from R_{l-1}
__global__ void k_box_fill(int level, int off, int ncell, const uint64_t* __restrict__ cells,
                           const uint64_t* __restrict__ Rl, int nRl, int off_next,
                           const uint64_t* __restrict__ cells_prev, int ncell_prev, int off_prev,
                           const uint64_t* __restrict__ pkeys, int64_t N, Geo g, BoxArrays B) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell) return;
    int b = off + i;
    uint64_t key = cells[i];
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
    int64_t r = (nRl > 0) ? find_u64(Rl, nRl, key) : -1;
    B.child0[b] = (r >= 0) ? off_next + 8 * (int)r : -1;
    if (level == 0) {
        B.parent[b] = -1;
    } else {
        int64_t pi = find_u64(cells_prev, ncell_prev, key >> 3);
        B.parent[b] = (pi >= 0) ? off_prev + (int)pi : -1;
    }
}

// non-leaf list: boxes whose key is in R_l, in R_l order
__global__ void k_nonleaf_list(int nRl, const uint64_t* __restrict__ Rl, const uint64_t* __restrict__ cells,
                               int ncell, int off, int nl_off, int* __restrict__ nl_box, int* __restrict__ nl_of_box) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nRl) return;
    int64_t pos = find_u64(cells, ncell, Rl[k]);
    int b = off + (int)pos;
    nl_box[nl_off + k] = b;
    nl_of_box[b] = nl_off + k;
}

// per-level arrays of the forest, passed by value to the all-level kernels below
struct LevelSet {
    const uint64_t* cells[kMaxLevels + 1];   // sorted cell keys of each level
    const uint64_t* R[kMaxLevels + 1];       // sorted non-leaf subset of each level
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

// k_box_fill for every level in one launch
__global__ void k_box_fill_all(LevelSet ls, int nb, const uint64_t* __restrict__ pkeys, int64_t N, Geo g,
                               BoxArrays B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int level = level_of(ls.off, ls.nlev, b);
    const int i = b - ls.off[level];
    const uint64_t key = ls.cells[level][i];
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
    B.nl[b] = (r >= 0) ? ls.nl_off[level] + (int)r : -1;
    if (level == 0) {
        B.parent[b] = -1;
    } else {
        const int np = ls.off[level] - ls.off[level - 1];
        const int64_t pi = find_u64(ls.cells[level - 1], np, key >> 3);
        B.parent[b] = (pi >= 0) ? ls.off[level - 1] + (int)pi : -1;
    }
}

// non-leaf list of every level in one launch: nl_box[nl_off_l + k] = box of R_l[k]
__global__ void k_nonleaf_all(LevelSet ls, int n_nl, int* __restrict__ nl_box) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nl) return;
    const int l = level_of(ls.nl_off, ls.nlev, t);
    const int k = t - ls.nl_off[l];
    const int ncell = ls.off[l + 1] - ls.off[l];
    nl_box[t] = ls.off[l] + (int)find_u64(ls.cells[l], ncell, ls.R[l][k]);
}

// colleague table: coll[b * 27 + d] = box at the same level with offset d, or -1
__global__ void k_colleagues(int nb, const int* __restrict__ level, const int* __restrict__ ixa,
                             const uint64_t* __restrict__ keys, const int* __restrict__ level_off,
                             const int* __restrict__ level_cnt, Geo g, int* __restrict__ coll) {
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
        int64_t pos = find_u64(keys + level_off[l], level_cnt[l], k);
        if (pos >= 0) res = level_off[l] + (int)pos;
    }
    coll[t] = res;
}

// leaves holding points
__global__ void k_leaf_flags(int nb, const int* __restrict__ child0, const int* __restrict__ start,
                             const int* __restrict__ end, int* __restrict__ flags, int* __restrict__ iota) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    flags[b] = (child0[b] < 0 && end[b] > start[b]) ? 1 : 0;
    iota[b] = b;
}

// Direct list of target leaf T (telescoping recursion of the split, Eqs. multilevel_ks,
// u_four_partsDP, Sec. 3.1.5):
//   (a) for j < level(T): leaf colleagues C of T's level-j ancestor, kernel K_R(nu_j);
//   (b) every colleague C of T (leaf or not: all points below it), kernel K_R(nu_level(T)).
// Entry = {start, end, packed shifts and level, unused}.
struct DirectEntry { int start, end, code, pad; };

__device__ __forceinline__ int pack_code(const int sh[3], int level) {
    return (sh[0] + 1) | ((sh[1] + 1) << 2) | ((sh[2] + 1) << 4) | (level << 6);
}

template <bool FILL>
__global__ void k_direct(int cap, const int* __restrict__ nleaf_dev, const int* __restrict__ leaves, BoxArrays B,
                         Geo g, int* __restrict__ counts, const int* __restrict__ offs, DirectEntry* __restrict__ out,
                         unsigned long long* __restrict__ npairs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    if (i >= nleaf_dev[0]) {
        if (!FILL) counts[i] = 0;
        return;
    }
    int T = leaves[i];
    int lT = B.level[T];
    int cnt = 0;
    long long pairs = 0;
    int pos = FILL ? offs[i] : 0;
    int nt = B.end[T] - B.start[T];
    // ancestors A_j, j = lT-1 .. 0
    int A = B.parent[T];
    for (int j = lT - 1; j >= 0; --j) {
        int ix[3] = {B.ix[3 * A], B.ix[3 * A + 1], B.ix[3 * A + 2]};
        for (int d = 0; d < 27; ++d) {
            int C = B.coll[A * 27 + d];
            if (C < 0 || B.child0[C] >= 0 || B.end[C] <= B.start[C]) continue;
            if (FILL) {
                int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1}, nbx[3], sh[3];
                neighbour(g, j, ix, dd, nbx, sh);
                out[pos++] = {B.start[C], B.end[C], pack_code(sh, j), 0};
            } else {
                ++cnt;
                pairs += (long long)(B.end[C] - B.start[C]) * nt;
            }
        }
        A = B.parent[A];
    }
    {
        int ix[3] = {B.ix[3 * T], B.ix[3 * T + 1], B.ix[3 * T + 2]};
        for (int d = 0; d < 27; ++d) {
            int C = B.coll[T * 27 + d];
            if (C < 0 || B.end[C] <= B.start[C]) continue;
            if (FILL) {
                int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1}, nbx[3], sh[3];
                neighbour(g, lT, ix, dd, nbx, sh);
                out[pos++] = {B.start[C], B.end[C], pack_code(sh, lT), 0};
            } else {
                ++cnt;
                pairs += (long long)(B.end[C] - B.start[C]) * nt;
            }
        }
    }
    if (!FILL) {
        counts[i] = cnt;
        atomicAdd(npairs, (unsigned long long)pairs);
    }
}

}  // namespace dmk
