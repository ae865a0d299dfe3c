// Evaluation kernels: upward pass (Sec. 3.1.2), root far field (Sec. 4.3, 5.3), plane-wave
// difference-kernel interactions (Sec. 2.3 Eq. Dl_int_discr, Sec. 3.1.4), Chebyshev shift to
// children (Sec. 3.1.4) and the leaf stage (Sec. 3.1.5, Sec. 2.4).
//
// Per-box tensors are stored x-major: t[(j1 * p + j2) * p + j3], j1 the x node index.
// Work buffers come from dynamic shared memory when they fit, else from a per-CTA slice of a
// global scratch array (the same code through a generic pointer).
#pragma once
#include "dmk_tree.cuh"

namespace dmk {

extern __shared__ __align__(16) unsigned char dsmem[];

__device__ __forceinline__ unsigned char* work_base(unsigned char* scratch, size_t per_cta, int use_smem) {
    return use_smem ? dsmem : scratch + (size_t)blockIdx.x * per_cta;
}

// Lagrange basis on first-kind Chebyshev nodes by the barycentric formula (nodes exact hits -> delta)
template <class T>
__device__ __forceinline__ void lagrange_row(T xi, const T* nodes, const T* bary, int p, T* out) {
    T den = 0;
    int hit = -1;
    for (int a = 0; a < p; ++a) {
        T d = xi - nodes[a];
        if (d == T(0)) hit = a;
        den += bary[a] / d;
    }
    if (hit >= 0) {
        for (int a = 0; a < p; ++a) out[a] = (a == hit) ? T(1) : T(0);
        return;
    }
    T inv = T(1) / den;
    for (int a = 0; a < p; ++a) out[a] = bary[a] / (xi - nodes[a]) * inv;
}

// ------------------------------------------------------------------------------------------
// Leaf anterpolation (Sec. 3.1.2): proxy(j1,j2,j3) = sum_s rho_s l_j1(xi_s) l_j2(eta_s) l_j3(zeta_s).
// Sources in chunks of kAnterpChunk: one thread per (source, axis) builds the Lagrange row
// (barycentric form, zero-padded to MAXP, the x row scaled by the strength); then one thread per
// (j2, j3) accumulates the p values over j1 in registers, reading the x rows as vectors.
constexpr int kAnterpChunk = 128;

template <class T>
__device__ __forceinline__ void lagrange_row_padded(T xi, const T* nodes, const T* bary, int p, int maxp, T scale,
                                                    T* out) {
    T den = 0;
    int hit = -1;
    for (int a = 0; a < p; ++a) {
        const T d = xi - nodes[a];
        if (d == T(0)) hit = a;
        const T w = bary[a] / d;
        out[a] = w;
        den += w;
    }
    if (hit >= 0) {
        for (int a = 0; a < p; ++a) out[a] = (a == hit) ? scale : T(0);
    } else {
        const T f = scale / den;
        for (int a = 0; a < p; ++a) out[a] *= f;
    }
    for (int a = p; a < maxp; ++a) out[a] = T(0);
}

template <class T, int MAXP>
__global__ void __launch_bounds__(MAXP <= 24 ? (MAXP * MAXP + 31) / 32 * 32 : 512, (MAXP <= 24 && sizeof(T) == 4) ? 2 : 1)
    k_anterp(const int* __restrict__ nleaf_dev, const int* __restrict__ leaves, BoxArrays B,
                                                 const double* __restrict__ xs, int64_t N,
                                                 const double* __restrict__ rs, Tab<T> tab, double s,
                                                 T* __restrict__ proxy, const int* __restrict__ perm,
                                                 int64_t n_orig) {
    static_assert(MAXP % 4 == 0, "rows are read as four-vectors");
    const int p = tab.p, p2 = p * p, drho = tab.d_rho;
    constexpr int PC = kAnterpChunk;
    T* lx = reinterpret_cast<T*>(dsmem);
    T* ly = lx + PC * MAXP;
    T* lz = ly + PC * MAXP;
    const int nleaf = *nleaf_dev;
    for (int li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const int box = leaves[li];
        const int l = B.level[box];
        const double r = s / (double)(1 << l), half = 0.5 * r;
        const double c[3] = {(B.ix[3 * box] + 0.5) * r, (B.ix[3 * box + 1] + 0.5) * r, (B.ix[3 * box + 2] + 0.5) * r};
        const int st = B.start[box], en = B.end[box];
        for (int a = 0; a < drho; ++a) {
            for (int pair0 = 0; pair0 < p2; pair0 += blockDim.x) {
                const int pair = pair0 + threadIdx.x;
                const bool active = pair < p2;
                const int jb = active ? pair / p : 0, jc = active ? pair % p : 0;
                T acc[MAXP];
#pragma unroll
                for (int j = 0; j < MAXP; ++j) acc[j] = 0;
                for (int s0 = st; s0 < en; s0 += PC) {
                    const int ns = min(PC, en - s0);
                    __syncthreads();
                    for (int u = threadIdx.x; u < 3 * ns; u += blockDim.x) {
                        const int ax = u / ns, pt = u - ax * ns;
                        const double xi = (xs[ax * N + s0 + pt] - c[ax]) / half;
                        T* row = (ax == 0 ? lx : (ax == 1 ? ly : lz)) + pt * MAXP;
                        // with perm: only the points perm < n_orig (the sources inside Omega)
                        const bool use = !perm || perm[s0 + pt] < n_orig;
                        const T wgt = (ax == 0) ? (use ? (T)rs[(int64_t)(s0 + pt) * drho + a] : T(0)) : T(1);
                        lagrange_row_padded<T>((T)xi, tab.nodes, tab.bary, p, MAXP, wgt, row);
                    }
                    __syncthreads();
                    if (active) {
                        for (int pt = 0; pt < ns; ++pt) {
                            const T t = ly[pt * MAXP + jb] * lz[pt * MAXP + jc];
                            const Quad<T>* rx = reinterpret_cast<const Quad<T>*>(lx + pt * MAXP);
#pragma unroll
                            for (int q = 0; q < MAXP / 4; ++q) {
                                const Quad<T> v = rx[q];
                                acc[4 * q] = fma(v.x, t, acc[4 * q]);
                                acc[4 * q + 1] = fma(v.y, t, acc[4 * q + 1]);
                                acc[4 * q + 2] = fma(v.z, t, acc[4 * q + 2]);
                                acc[4 * q + 3] = fma(v.w, t, acc[4 * q + 3]);
                            }
                        }
                    }
                }
                if (active) {
                    T* out = proxy + ((size_t)box * drho + a) * p * p2;
#pragma unroll
                    for (int j = 0; j < MAXP; ++j)
                        if (j < p) out[j * p2 + pair] = acc[j];
                }
            }
        }
        __syncthreads();
    }
}

// Anterpolation with two (j2, j3) pairs per thread, (j2, j3) and (j2 + ceil(p/2), j3), which
// share the z row value and every x row load: 40 FMA per source for 3 + MAXP/4 shared-memory
// loads.  Threads: ceil(p/2) p.
template <class T, int MAXP>
__global__ void __launch_bounds__((MAXP / 2 * MAXP + 31) / 32 * 32, sizeof(T) == 4 ? 2 : 1)
    k_anterp2(const int* __restrict__ nleaf_dev, const int* __restrict__ leaves, BoxArrays B, const double* __restrict__ xs, int64_t N,
              const double* __restrict__ rs, Tab<T> tab, double s, T* __restrict__ proxy) {
    static_assert(MAXP % 4 == 0, "rows are read as four-vectors");
    const int p = tab.p, p2 = p * p, drho = tab.d_rho, hq = (p + 1) / 2;
    constexpr int PC = kAnterpChunk;
    T* lx = reinterpret_cast<T*>(dsmem);
    T* ly = lx + PC * MAXP;
    T* lz = ly + PC * MAXP;
    const int q = threadIdx.x;
    const bool active = q < hq * p;
    const int jb = active ? q / p : 0, jc = active ? q % p : 0;
    const bool second = active && jb + hq < p;
    const int nleaf = *nleaf_dev;
    for (int li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const int box = leaves[li];
        const int l = B.level[box];
        const double r = s / (double)(1 << l), half = 0.5 * r;
        const double c[3] = {(B.ix[3 * box] + 0.5) * r, (B.ix[3 * box + 1] + 0.5) * r, (B.ix[3 * box + 2] + 0.5) * r};
        const int st = B.start[box], en = B.end[box];
        for (int a = 0; a < drho; ++a) {
            T acc[MAXP], acc2[MAXP];
#pragma unroll
            for (int j = 0; j < MAXP; ++j) { acc[j] = 0; acc2[j] = 0; }
            for (int s0 = st; s0 < en; s0 += PC) {
                const int ns = min(PC, en - s0);
                __syncthreads();
                for (int u = threadIdx.x; u < 3 * ns; u += blockDim.x) {
                    const int ax = u / ns, pt = u - ax * ns;
                    const double xi = (xs[ax * N + s0 + pt] - c[ax]) / half;
                    T* row = (ax == 0 ? lx : (ax == 1 ? ly : lz)) + pt * MAXP;
                    const T wgt = (ax == 0) ? (T)rs[(int64_t)(s0 + pt) * drho + a] : T(1);
                    lagrange_row_padded<T>((T)xi, tab.nodes, tab.bary, p, MAXP, wgt, row);
                }
                __syncthreads();
                if (active) {
                    for (int pt = 0; pt < ns; ++pt) {
                        const T z = lz[pt * MAXP + jc];
                        const T t = ly[pt * MAXP + jb] * z;
                        const T t2 = second ? ly[pt * MAXP + jb + hq] * z : T(0);
                        const Quad<T>* rx = reinterpret_cast<const Quad<T>*>(lx + pt * MAXP);
#pragma unroll
                        for (int k = 0; k < MAXP / 4; ++k) {
                            const Quad<T> v = rx[k];
                            acc[4 * k] = fma(v.x, t, acc[4 * k]);
                            acc[4 * k + 1] = fma(v.y, t, acc[4 * k + 1]);
                            acc[4 * k + 2] = fma(v.z, t, acc[4 * k + 2]);
                            acc[4 * k + 3] = fma(v.w, t, acc[4 * k + 3]);
                            acc2[4 * k] = fma(v.x, t2, acc2[4 * k]);
                            acc2[4 * k + 1] = fma(v.y, t2, acc2[4 * k + 1]);
                            acc2[4 * k + 2] = fma(v.z, t2, acc2[4 * k + 2]);
                            acc2[4 * k + 3] = fma(v.w, t2, acc2[4 * k + 3]);
                        }
                    }
                }
            }
            if (active) {
                T* out = proxy + ((size_t)box * drho + a) * p * p2;
                const int pair = jb * p + jc, pair2 = (jb + hq) * p + jc;
#pragma unroll
                for (int j = 0; j < MAXP; ++j)
                    if (j < p) {
                        out[j * p2 + pair] = acc[j];
                        if (second) out[j * p2 + pair2] = acc2[j];
                    }
            }
        }
        __syncthreads();
    }
}

// Anterpolation as a register-tiled product (FP32 path), onto the grid of the box that needs a
// proxy: proxy_P[a][j1][(j2, j3)] = sum_s rho_{s,a} l_j1(xi_s) l_j2(eta_s) l_j3(zeta_s), xi the
// coordinates relative to P.  Only non-leaf boxes (plane waves, upward pass) and the cubes
// (structure factor) use proxies, so the sources of a leaf are anterpolated straight onto the
// grid of its parent: by the interpolation identity sum_j l^C_j(x) l^P_a(y^C_j) = l^P_a(x)
// (degree p - 1 reproduced at the child's p nodes) this equals the leaf proxy followed by the
// child-to-parent interpolation of Sec. 3.1.2 and spares that interpolation.  Work item: a
// non-leaf box with at least one leaf child (the sources of its leaf children), or a cube that
// is a leaf (its own sources); k_up_cluster adds the non-leaf children afterwards.
//   The Lagrange rows of up to ROWS sources (gathered over the leaf children) are computed
// once and kept in shared memory with the strengths, for every component; each thread owns a
// tile of 4 consecutive j1 x every j3 (TN = MAXP, zero rows beyond p) at one (a, j2) and per
// source forms w = rho_a l_j2 l_j1[4] (5 multiplies) and does 4 TN multiply-adds from 3 + TN/4
// shared-memory reads.  Tiles beyond the block's threads are taken in passes over the same rows.
constexpr int kAntRows = 256;      // sources whose Lagrange rows are held at once (parent items)
constexpr int kAntRowsLeaf = 128;  // the same for leaf items (at most n_s sources, often ~100):
                                   // half the shared memory, more resident blocks
constexpr int kAntThreads = 256;

template <int MAXP, int ROWS>
struct AntSmem {
    static constexpr size_t lx = 0;                                         // float [ROWS][MAXP]
    static constexpr size_t ly = lx + (size_t)ROWS * MAXP * 4;
    static constexpr size_t lz = ly + (size_t)ROWS * MAXP * 4;
    static constexpr size_t rho = lz + (size_t)ROWS * MAXP * 4;            // float [ROWS][9]
    static constexpr size_t bytes = rho + (size_t)ROWS * 9 * 4;
};

//   With leaf_list (few parents: too few work items for the GPU), the items are the leaves
// themselves, each anterpolated onto its parent's grid (a cube that is a leaf: its own) into the
// leaf's own proxy slot; k_leaf_partials then sums each parent's leaf children in child order.
// With leaf_list and !to_parent every leaf is anterpolated onto its own grid (the upward pass
// then takes every child).
template <int MAXP, int TN, int ROWS>
__global__ void __launch_bounds__(kAntThreads, 2)
    k_anterp3(int n_nl, const int* __restrict__ nl_box, int n_root, BoxArrays B, const double* __restrict__ xs,
              int64_t N, const double* __restrict__ rs, Tab<float> tab, double s, float* __restrict__ proxy,
              const int* __restrict__ leaf_list, const int* __restrict__ nleaf_dev, int to_parent) {
    static_assert(MAXP % 4 == 0 && TN % 4 == 0 && TN <= MAXP, "vector reads");
    using S = AntSmem<MAXP, ROWS>;
    const int p = tab.p, p2 = p * p, p3 = p2 * p, drho = tab.d_rho;
    const int nj = (p + 3) / 4, ng = (p + TN - 1) / TN, ntile = drho * nj * p * ng;
    float* lx = reinterpret_cast<float*>(dsmem + S::lx);
    float* ly = reinterpret_cast<float*>(dsmem + S::ly);
    float* lz = reinterpret_cast<float*>(dsmem + S::lz);
    float* rh = reinterpret_cast<float*>(dsmem + S::rho);
    __shared__ int rng[8][2];
    __shared__ int nrng;
    const int n_items = leaf_list ? *nleaf_dev : n_nl + n_root;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        int box;
        __syncthreads();
        if (leaf_list) {
            box = leaf_list[item];
            if (threadIdx.x == 0) {
                nrng = 1;
                rng[0][0] = B.start[box];
                rng[0][1] = B.end[box];
            }
        } else if (item < n_nl) {
            box = nl_box[item];
            if (threadIdx.x == 0) {
                int k = 0;
                const int c0 = B.child0[box];
                for (int o = 0; o < 8; ++o)
                    if (B.child0[c0 + o] < 0) { rng[k][0] = B.start[c0 + o]; rng[k][1] = B.end[c0 + o]; ++k; }
                nrng = k;
            }
        } else {
            box = item - n_nl;                     // cube index = box index at level 0
            if (threadIdx.x == 0) {
                nrng = (B.child0[box] < 0) ? 1 : 0;
                rng[0][0] = B.start[box];
                rng[0][1] = B.end[box];
            }
        }
        __syncthreads();
        const int nr = nrng;
        if (nr == 0) continue;                     // uniform over the block
        // the grid the sources go onto: the box's own, or (split leaf items) its parent's
        const int gb = (leaf_list && to_parent && B.parent[box] >= 0) ? B.parent[box] : box;
        const int l = B.level[gb];
        const double r = s / (double)(1 << l), half = 0.5 * r, ihalf = 1.0 / half;
        const double cx = (B.ix[3 * gb] + 0.5) * r, cy = (B.ix[3 * gb + 1] + 0.5) * r,
                     cz = (B.ix[3 * gb + 2] + 0.5) * r;
        float* outb = proxy + (size_t)box * drho * p3;
        // the sources of the ranges in super-chunks of ROWS (cursor: range ri, position pos)
        int ri = 0, pos = rng[0][0];
        bool first = true;
        while (true) {
            // gather the next super-chunk's point indices (uniform cursor logic)
            int ns = 0;
            int cr = ri, cp = pos;
            __syncthreads();
            while (cr < nr && ns < ROWS) {
                const int take = min(ROWS - ns, rng[cr][1] - cp);
                for (int u = threadIdx.x; u < 3 * take; u += blockDim.x) {
                    const int ax = u / take, pt = u - ax * take;
                    const double c = ax == 0 ? cx : (ax == 1 ? cy : cz);
                    const double xi = (xs[ax * N + cp + pt] - c) * ihalf;
                    float* row = (ax == 0 ? lx : (ax == 1 ? ly : lz)) + (ns + pt) * MAXP;
                    lagrange_row_padded<float>((float)xi, tab.nodes, tab.bary, p, MAXP, 1.0f, row);
                }
                for (int u = threadIdx.x; u < take * drho; u += blockDim.x)
                    rh[ns * drho + u] = (float)rs[(int64_t)cp * drho + u];
                ns += take;
                cp += take;
                if (cp >= rng[cr][1]) {
                    ++cr;
                    if (cr < nr) cp = rng[cr][0];
                }
            }
            ri = cr;
            pos = cp;
            __syncthreads();
            for (int tile = threadIdx.x; tile < ntile; tile += blockDim.x) {
                // tile -> (component a, row block jt, j2, column group g)
                const int g = tile % ng, r1 = tile / ng;
                const int j2 = r1 % p, r2 = r1 / p;
                const int jt = r2 % nj, a = r2 / nj;
                const int j30 = g * TN;
                float acc[4][TN];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < TN; ++q) acc[i][q] = 0.f;
                const float* px = lx + 4 * jt;
                const float* py = ly + j2;
                const float* pz = lz + j30;
                const float* pr = rh + a;
#pragma unroll 1
                for (int k = 0; k < ns; ++k) {
                    const float4 xv = *reinterpret_cast<const float4*>(px + k * MAXP);
                    const float f = pr[k * drho] * py[k * MAXP];
                    const float w[4] = {xv.x * f, xv.y * f, xv.z * f, xv.w * f};
                    const float4* zr = reinterpret_cast<const float4*>(pz + k * MAXP);
#pragma unroll
                    for (int q = 0; q < TN / 4; ++q) {
                        const float4 zv = zr[q];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            acc[i][4 * q] = fmaf(w[i], zv.x, acc[i][4 * q]);
                            acc[i][4 * q + 1] = fmaf(w[i], zv.y, acc[i][4 * q + 1]);
                            acc[i][4 * q + 2] = fmaf(w[i], zv.z, acc[i][4 * q + 2]);
                            acc[i][4 * q + 3] = fmaf(w[i], zv.w, acc[i][4 * q + 3]);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int j1 = 4 * jt + i;
                    if (j1 < p) {
                        float* o = outb + ((size_t)a * p + j1) * p2 + j2 * p + j30;
#pragma unroll
                        for (int q = 0; q < TN; ++q)
                            if (j30 + q < p) o[q] = first ? acc[i][q] : o[q] + acc[i][q];
                    }
                }
            }
            first = false;
            if (ri >= nr) break;
        }
    }
}

template <int MAXP>
inline size_t anterp3_smem(bool leaf_items) {
    return leaf_items ? AntSmem<MAXP, kAntRowsLeaf>::bytes : AntSmem<MAXP, kAntRows>::bytes;
}

// The split form of the direct upward path: every non-leaf box with leaf children gets the sum,
// in child order, of its non-empty leaf children's partial grids (their sources on its grid,
// k_anterp3 with leaf_list and to_parent), stored as its proxy; per_box = d_rho p^3.  Boxes
// without leaf children are left to k_up_cluster.
template <class T>
__global__ void k_leaf_partials(int n_nl, const int* __restrict__ nl_box, BoxArrays B, int per_box,
                                T* __restrict__ proxy) {
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)n_nl * per_box) return;
    const int item = (int)(id / per_box), e = (int)(id - (int64_t)item * per_box);
    const int P = nl_box[item], c0 = B.child0[P];
    T v = 0;
    bool any = false;
    for (int o = 0; o < 8; ++o) {
        const int c = c0 + o;
        if (B.child0[c] >= 0) continue;
        any = true;
        if (B.end[c] > B.start[c]) v += proxy[(size_t)c * per_box + e];
    }
    if (any) proxy[(size_t)P * per_box + e] = v;
}

// ------------------------------------------------------------------------------------------
// Upward pass child -> parent (Sec. 3.1.2): parent += sum_children (I^T x I^T x I^T) child,
// I[o][j_child][a_parent] = l_a(child node j in parent coordinates).
template <class T>
__global__ void k_upward(int n, const int* __restrict__ nl_box, BoxArrays B, Tab<T> tab, T* __restrict__ proxy,
                         unsigned char* scratch, size_t per_cta, int use_smem) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, drho = tab.d_rho;
    T* t1 = reinterpret_cast<T*>(work_base(scratch, per_cta, use_smem));
    T* t2 = t1 + p3;
    T* acc = t2 + p3;
    for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const int P = nl_box[bi];
        const int c0 = B.child0[P];
        for (int a = 0; a < drho; ++a) {
            for (int e = threadIdx.x; e < p3; e += blockDim.x) acc[e] = 0;
            for (int o = 0; o < 8; ++o) {
                const T* ch = proxy + ((size_t)(c0 + o) * drho + a) * p3;
                const T* Iz = tab.Ioct + ((o >> 2) & 1) * p2;
                const T* Iy = tab.Ioct + ((o >> 1) & 1) * p2;
                const T* Ix = tab.Ioct + (o & 1) * p2;
                __syncthreads();
                for (int e = threadIdx.x; e < p3; e += blockDim.x) {      // contract z
                    const int i12 = e / p, cc = e % p;
                    T v = 0;
                    for (int k = 0; k < p; ++k) v = fma(ch[i12 * p + k], Iz[k * p + cc], v);
                    t1[e] = v;
                }
                __syncthreads();
                for (int e = threadIdx.x; e < p3; e += blockDim.x) {      // contract y
                    const int i1 = e / p2, bb = (e / p) % p, cc = e % p;
                    T v = 0;
                    for (int k = 0; k < p; ++k) v = fma(t1[(i1 * p + k) * p + cc], Iy[k * p + bb], v);
                    t2[e] = v;
                }
                __syncthreads();
                for (int e = threadIdx.x; e < p3; e += blockDim.x) {      // contract x
                    const int aa = e / p2, r23 = e % p2;
                    T v = acc[e];
                    for (int k = 0; k < p; ++k) v = fma(t2[k * p2 + r23], Ix[k * p + aa], v);
                    acc[e] = v;
                }
            }
            __syncthreads();
            T* out = proxy + ((size_t)P * drho + a) * p3;
            for (int e = threadIdx.x; e < p3; e += blockDim.x) out[e] = acc[e];
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------------------------------
// Shift to children (Sec. 3.1.4): local(child) += (I x I x I) local(parent)
template <class T>
__global__ void k_shift(int n, const int* __restrict__ nl_box, BoxArrays B, Tab<T> tab, T* __restrict__ local,
                        unsigned char* scratch, size_t per_cta, int use_smem) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, du = tab.d_u;
    T* t1 = reinterpret_cast<T*>(work_base(scratch, per_cta, use_smem));
    T* t2 = t1 + p3;
    for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const int P = nl_box[bi];
        const int c0 = B.child0[P];
        for (int j = 0; j < du; ++j) {
            const T* par = local + ((size_t)P * du + j) * p3;
            for (int o = 0; o < 8; ++o) {
                const T* Iz = tab.Ioct + ((o >> 2) & 1) * p2;
                const T* Iy = tab.Ioct + ((o >> 1) & 1) * p2;
                const T* Ix = tab.Ioct + (o & 1) * p2;
                __syncthreads();
                for (int e = threadIdx.x; e < p3; e += blockDim.x) {
                    const int i12 = e / p, cc = e % p;
                    T v = 0;
                    for (int k = 0; k < p; ++k) v = fma(Iz[cc * p + k], par[i12 * p + k], v);
                    t1[e] = v;
                }
                __syncthreads();
                for (int e = threadIdx.x; e < p3; e += blockDim.x) {
                    const int i1 = e / p2, bb = (e / p) % p, cc = e % p;
                    T v = 0;
                    for (int k = 0; k < p; ++k) v = fma(Iy[bb * p + k], t1[(i1 * p + k) * p + cc], v);
                    t2[e] = v;
                }
                __syncthreads();
                T* ch = local + ((size_t)(c0 + o) * du + j) * p3;
                for (int e = threadIdx.x; e < p3; e += blockDim.x) {
                    const int aa = e / p2, r23 = e % p2;
                    T v = 0;
                    for (int k = 0; k < p; ++k) v = fma(Ix[aa * p + k], t2[k * p2 + r23], v);
                    ch[e] += v;
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Plane-wave outgoing expansions (Sec. 3.1.4, Eq. Dl_int_discr): for every non-leaf box,
// W(m) = sum_j proxy(j) exp(-i h m . y_j); h y_j = (pi/3) m eta_j at every level.  Real input,
// so only m3 >= 0 is stored: W[nl][a][(m1 * NF + m2) * nfh + m3].
template <class T>
__global__ void k_pwout(int n, const int* __restrict__ nl_box, Tab<T> tab, const T* __restrict__ proxy,
                        Cx<T>* __restrict__ W, unsigned char* scratch, size_t per_cta, int use_smem) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, drho = tab.d_rho;
    const int nf = tab.nf, NF = tab.NF, nfh = tab.nfh;
    const int nW = NF * NF * nfh;
    Cx<T>* A1 = reinterpret_cast<Cx<T>*>(work_base(scratch, per_cta, use_smem));
    Cx<T>* A2 = A1 + p2 * nfh;
    for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const int box = nl_box[bi];
        for (int a = 0; a < drho; ++a) {
            const T* pr = proxy + ((size_t)box * drho + a) * p3;
            __syncthreads();
            for (int e = threadIdx.x; e < p2 * nfh; e += blockDim.x) {   // j3 -> m3 (>= 0)
                const int i12 = e / nfh, m3 = e % nfh;
                const Cx<T>* Er = tab.E + (nf + m3) * p;
                Cx<T> v = {0, 0};
                for (int k = 0; k < p; ++k) cfmar(v, Er[k], pr[i12 * p + k]);
                A1[e] = v;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < p * NF * nfh; e += blockDim.x) {   // j2 -> m2
                const int i1 = e / (NF * nfh), m2 = (e / nfh) % NF, m3 = e % nfh;
                const Cx<T>* Er = tab.E + m2 * p;
                Cx<T> v = {0, 0};
                for (int k = 0; k < p; ++k) cfma(v, Er[k], A1[(i1 * p + k) * nfh + m3]);
                A2[e] = v;
            }
            __syncthreads();
            Cx<T>* out = W + ((size_t)bi * drho + a) * nW;
            for (int e = threadIdx.x; e < nW; e += blockDim.x) {           // j1 -> m1
                const int m1 = e / (NF * nfh), r = e % (NF * nfh);
                const Cx<T>* Er = tab.E + m1 * p;
                Cx<T> v = {0, 0};
                for (int k = 0; k < p; ++k) cfma(v, Er[k], A2[k * NF * nfh + r]);
                out[e] = v;
            }
        }
        __syncthreads();
    }
}

// operator symbol of the kernel on the integer wave vector m (App. B): out[j][a] = op_ja(m) * V_a
template <class T>
__device__ __forceinline__ void apply_op(int kernel, const T m[3], const Cx<T>* V, Cx<T>* out) {
    if (kernel == DMK_LAPLACE) {
        out[0] = V[0];
    } else if (kernel == DMK_STOKESLET) {
        const T m2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
        Cx<T> md = {0, 0};
        for (int l = 0; l < 3; ++l) cfmar(md, V[l], m[l]);
        for (int j = 0; j < 3; ++j) out[j] = {m2 * V[j].x - m[j] * md.x, m2 * V[j].y - m[j] * md.y};
    } else if (kernel == DMK_STRESSLET) {
        // i [ (m_m d_jl + m_l d_mj + m_j d_lm) |m|^2 - 2 m_j m_l m_m ] Q_lm
        const T m2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
        Cx<T> Qm[3], QTm[3], tr = {V[0].x + V[4].x + V[8].x, V[0].y + V[4].y + V[8].y}, mQm = {0, 0};
        for (int j = 0; j < 3; ++j) {
            Qm[j] = {0, 0};
            QTm[j] = {0, 0};
            for (int k = 0; k < 3; ++k) {
                cfmar(Qm[j], V[j * 3 + k], m[k]);
                cfmar(QTm[j], V[k * 3 + j], m[k]);
            }
        }
        for (int j = 0; j < 3; ++j) cfmar(mQm, Qm[j], m[j]);
        for (int j = 0; j < 3; ++j) {
            Cx<T> v = {m2 * (Qm[j].x + QTm[j].x + m[j] * tr.x) - 2 * m[j] * mQm.x,
                       m2 * (Qm[j].y + QTm[j].y + m[j] * tr.y) - 2 * m[j] * mQm.y};
            out[j] = {-v.y, v.x};     // times i
        }
    } else {
        // rotlet: -1/2 i eps_jlm m_m tau_l = -1/2 i (tau x m)_j
        Cx<T> c[3];
        c[0] = {V[1].x * m[2] - V[2].x * m[1], V[1].y * m[2] - V[2].y * m[1]};
        c[1] = {V[2].x * m[0] - V[0].x * m[2], V[2].y * m[0] - V[0].y * m[2]};
        c[2] = {V[0].x * m[1] - V[1].x * m[0], V[0].y * m[1] - V[1].y * m[0]};
        for (int j = 0; j < 3; ++j) out[j] = {T(0.5) * c[j].y, T(-0.5) * c[j].x};
    }
}

// Translation over colleagues, symbol, incoming transform (Sec. 3.1.4): for non-leaf B,
//   V(m) = sum_{non-leaf colleague C at offset d} exp(-i (2 pi/3) m.d) W_C(m),
//   u_B(j) += Re sum_m 2^(a l) g(m) op(m) V(m) exp(+i (pi/3) m . eta_j).
template <class T>
__global__ void k_pwin(int n, const int* __restrict__ nl_box, BoxArrays B, Tab<T> tab, const Cx<T>* __restrict__ W,
                       T* __restrict__ local, unsigned char* scratch, size_t per_cta, int use_smem) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, drho = tab.d_rho, du = tab.d_u;
    const int nf = tab.nf, NF = tab.NF, nfh = tab.nfh;
    const int nW = NF * NF * nfh;
    Cx<T>* Vp = reinterpret_cast<Cx<T>*>(work_base(scratch, per_cta, use_smem));
    Cx<T>* B2 = Vp + du * nW;
    Cx<T>* B1 = B2 + p * NF * nfh;
    __shared__ int ncol;
    __shared__ int col_nl[27];
    __shared__ int col_d[27];
    const T c3 = T(-0.5), s3 = T(-0.86602540378443864676);   // exp(-i 2 pi/3)
    for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const int box = nl_box[bi];
        const int l = B.level[box];
        const T scale = (T)ldexp(1.0, tab.level_power * l);
        __syncthreads();
        if (threadIdx.x == 0) {
            int k = 0;
            for (int d = 0; d < 27; ++d) {
                const int C = B.coll[box * 27 + d];
                if (C >= 0 && B.nl[C] >= 0) { col_nl[k] = B.nl[C]; col_d[k] = d; ++k; }
            }
            ncol = k;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nW; e += blockDim.x) {
            const int i1 = e / (NF * nfh), i2 = (e / nfh) % NF, m3 = e % nfh;
            const int m1 = i1 - nf, m2 = i2 - nf;
            Cx<T> V[9];
            for (int a = 0; a < drho; ++a) V[a] = {0, 0};
            for (int k = 0; k < ncol; ++k) {
                const int d = col_d[k];
                const int dot = m1 * (d % 3 - 1) + m2 * ((d / 3) % 3 - 1) + m3 * (d / 9 - 1);
                const int r = ((dot % 3) + 3) % 3;
                const Cx<T> ph = (r == 0) ? Cx<T>{1, 0} : (r == 1 ? Cx<T>{c3, s3} : Cx<T>{c3, -s3});
                const Cx<T>* Wc = W + (size_t)col_nl[k] * drho * nW + e;
                for (int a = 0; a < drho; ++a) cfma(V[a], ph, Wc[(size_t)a * nW]);
            }
            const T g = scale * tab.gdiff[e];
            const T mv[3] = {(T)m1, (T)m2, (T)m3};
            Cx<T> out[3];
            apply_op<T>(tab.kernel, mv, V, out);
            for (int j = 0; j < du; ++j) Vp[(size_t)j * nW + e] = {g * out[j].x, g * out[j].y};
        }
        for (int j = 0; j < du; ++j) {
            __syncthreads();
            const Cx<T>* Vj = Vp + (size_t)j * nW;
            for (int e = threadIdx.x; e < p * NF * nfh; e += blockDim.x) {   // m1 -> j1
                const int i1 = e / (NF * nfh), r = e % (NF * nfh);
                Cx<T> v = {0, 0};
                for (int k = 0; k < NF; ++k) cfma(v, cconj(tab.E[k * p + i1]), Vj[k * NF * nfh + r]);
                B2[e] = v;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < p2 * nfh; e += blockDim.x) {       // m2 -> j2
                const int i1 = e / (p * nfh), i2 = (e / nfh) % p, m3 = e % nfh;
                Cx<T> v = {0, 0};
                for (int k = 0; k < NF; ++k) cfma(v, cconj(tab.E[k * p + i2]), B2[(i1 * NF + k) * nfh + m3]);
                B1[e] = v;
            }
            __syncthreads();
            T* u = local + ((size_t)box * du + j) * p3;
            for (int e = threadIdx.x; e < p3; e += blockDim.x) {             // m3 -> j3, real part
                const int i12 = e / p, i3 = e % p;
                T v = 0;
                for (int m3 = 0; m3 < nfh; ++m3) {
                    const Cx<T> f = cconj(tab.E[(nf + m3) * p + i3]);
                    const Cx<T> b = B1[i12 * nfh + m3];
                    const T re = f.x * b.x - f.y * b.y;
                    v += (m3 == 0 ? T(1) : T(2)) * re;
                }
                u[e] += v;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Root far field (Sec. 4.3 Eqs. structurefac and eval_tensor; Sec. 5.3 Eq. ewald_far_allP_discr), FP64.
struct RootTab {
    int n1, n2, n3, nmode;
    int Q[3];                    // cube-index DFT length per axis (1 without one)
    const double* kax[3];
    const Cx<double>* S[3];      // S_i[k * p + j] = exp(-i k (s/2) eta_j)
    const Cx<double>* W;         // nmode x du x drho
    const double* rconst;        // du x drho
    const double* nmod[3];       // per wavenumber k = 2 pi n / (Q_a s) of axis a: n mod Q_a
    const Cx<double>* roots[3];  // exp(2 pi i t / Q_a), t = 0..Q_a-1
};

// sum over cubes and apply the symbol: uhat[j][k] = sum_a W[k][j][a] sum_m chi_m,a(k)
__global__ void k_root_apply(int M, int drho, int du, RootTab rt, const Cx<double>* __restrict__ chi_part,
                             Cx<double>* __restrict__ uhat) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rt.nmode) return;
    Cx<double> chi[9];
    for (int a = 0; a < drho; ++a) {
        Cx<double> v = {0, 0};
        for (int m = 0; m < M; ++m) v = cadd(v, chi_part[((size_t)m * drho + a) * rt.nmode + k]);
        chi[a] = v;
    }
    for (int j = 0; j < du; ++j) {
        Cx<double> v = {0, 0};
        for (int a = 0; a < drho; ++a) cfma(v, rt.W[((size_t)k * du + j) * drho + a], chi[a]);
        uhat[(size_t)j * rt.nmode + k] = v;
    }
}

// Root far field spread over the whole GPU: every stage of the tensor-form sums of Eqs.
// structurefac and eval_tensor is its own launch with one thread per output
// element of all cubes and components, so that the FP64 work is not confined to one CTA per
// cube.  Scratch layout per job (cube m, component): B1 n1 x p^2, B2 n1 x n2 x p (forward);
// G nmode, C2 n1 x n2 x p, C1 n1 x p^2 (backward).
template <class T>
__global__ void k_root_fwd1(int jobs, int p, RootTab rt, const T* __restrict__ proxy, Cx<double>* __restrict__ B1) {
    const int p2 = p * p, p3 = p2 * p, per = rt.n1 * p2;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)jobs * per) return;
    const int job = (int)(id / per), e = (int)(id % per);
    const int i1 = e / p2, r = e % p2;
    const T* pr = proxy + (size_t)job * p3;
    Cx<double> v = {0, 0};
    for (int k = 0; k < p; ++k) cfmar(v, rt.S[0][i1 * p + k], (double)pr[k * p2 + r]);
    B1[id] = v;
}

__global__ void k_root_fwd2(int jobs, int p, RootTab rt, const Cx<double>* __restrict__ B1,
                            Cx<double>* __restrict__ B2) {
    const int p2 = p * p, n2 = rt.n2, per = rt.n1 * n2 * p;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)jobs * per) return;
    const int job = (int)(id / per), e = (int)(id % per);
    const int i1 = e / (n2 * p), i2 = (e / p) % n2, j3 = e % p;
    const Cx<double>* b = B1 + (size_t)job * rt.n1 * p2 + (size_t)i1 * p2 + j3;
    Cx<double> v = {0, 0};
    for (int k = 0; k < p; ++k) cfma(v, rt.S[1][i2 * p + k], b[k * p]);
    B2[id] = v;
}

__global__ void k_root_fwd3(int jobs, int drho, int p, Geo g, RootTab rt, const Cx<double>* __restrict__ B2,
                            Cx<double>* __restrict__ chi_part) {
    const int n2 = rt.n2, n3 = rt.n3, per = rt.nmode;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)jobs * per) return;
    const int job = (int)(id / per), e = (int)(id % per);
    const int m = job / drho;
    const int mc[3] = {m % g.M[0], (m / g.M[0]) % g.M[1], m / (g.M[0] * g.M[1])};
    const int i1 = e / (n2 * n3), i2 = (e / n3) % n2, i3 = e % n3;
    const Cx<double>* b = B2 + (size_t)job * rt.n1 * n2 * p + ((size_t)i1 * n2 + i2) * p;
    Cx<double> v = {0, 0};
    for (int k = 0; k < p; ++k) cfma(v, rt.S[2][i3 * p + k], b[k]);
    const double ph = -(rt.kax[0][i1] * (mc[0] + 0.5) * g.s + rt.kax[1][i2] * (mc[1] + 0.5) * g.s +
                        rt.kax[2][i3] * (mc[2] + 0.5) * g.s);
    double sn, cs;
    sincos(ph, &sn, &cs);
    chi_part[id] = cmul(v, Cx<double>{cs, sn});
}

__global__ void k_root_bwd0(int jobs, int du, Geo g, RootTab rt, const Cx<double>* __restrict__ uhat,
                            Cx<double>* __restrict__ G) {
    const int n2 = rt.n2, n3 = rt.n3, per = rt.nmode;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)jobs * per) return;
    const int job = (int)(id / per), e = (int)(id % per);
    const int m = job / du, j = job % du;
    const int mc[3] = {m % g.M[0], (m / g.M[0]) % g.M[1], m / (g.M[0] * g.M[1])};
    const int i1 = e / (n2 * n3), i2 = (e / n3) % n2, i3 = e % n3;
    const double ph = rt.kax[0][i1] * (mc[0] + 0.5) * g.s + rt.kax[1][i2] * (mc[1] + 0.5) * g.s +
                      rt.kax[2][i3] * (mc[2] + 0.5) * g.s;
    double sn, cs;
    sincos(ph, &sn, &cs);
    G[id] = cmul(uhat[(size_t)j * rt.nmode + e], Cx<double>{cs, sn});
}

__global__ void k_root_bwd1(int jobs, int p, RootTab rt, const Cx<double>* __restrict__ G,
                            Cx<double>* __restrict__ C2) {
    const int n3 = rt.n3, per = rt.n1 * rt.n2 * p;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)jobs * per) return;
    const int job = (int)(id / per), e = (int)(id % per);
    const int i12 = e / p, j3 = e % p;
    const Cx<double>* gg = G + (size_t)job * rt.nmode + (size_t)i12 * n3;
    Cx<double> v = {0, 0};
    for (int k = 0; k < n3; ++k) cfma(v, cconj(rt.S[2][k * p + j3]), gg[k]);
    C2[id] = v;
}

__global__ void k_root_bwd2(int jobs, int p, RootTab rt, const Cx<double>* __restrict__ C2,
                            Cx<double>* __restrict__ C1) {
    const int p2 = p * p, n2 = rt.n2, per = rt.n1 * p2;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)jobs * per) return;
    const int job = (int)(id / per), e = (int)(id % per);
    const int i1 = e / p2, j2 = (e / p) % p, j3 = e % p;
    const Cx<double>* c = C2 + (size_t)job * rt.n1 * n2 * p + (size_t)i1 * n2 * p + j3;
    Cx<double> v = {0, 0};
    for (int k = 0; k < n2; ++k) cfma(v, cconj(rt.S[1][k * p + j2]), c[k * p]);
    C1[id] = v;
}

template <class T>
__global__ void k_root_bwd3(int jobs, int du, int p, RootTab rt, const Cx<double>* __restrict__ C1,
                            const double* __restrict__ rho_sum, int drho, T* __restrict__ local, int add) {
    const int p2 = p * p, p3 = p2 * p;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)jobs * p3) return;
    const int job = (int)(id / p3), e = (int)(id % p3);
    const int j = job % du;
    const int j1 = e / p2, r = e % p2;
    const Cx<double>* c = C1 + (size_t)job * rt.n1 * p2 + r;
    double v = 0;
    for (int k = 0; k < rt.n1; ++k) {
        const Cx<double> f = cconj(rt.S[0][k * p + j1]);
        const Cx<double> b = c[(size_t)k * p2];
        v += f.x * b.x - f.y * b.y;
    }
    // add: a second root part, added to the first (whose write carried the constant)
    if (add) {
        local[(size_t)job * p3 + e] = (T)((double)local[(size_t)job * p3 + e] + v);
        return;
    }
    double cst = 0;
    if (rho_sum) for (int a = 0; a < drho; ++a) cst += rt.rconst[j * drho + a] * rho_sum[a];
    local[(size_t)job * p3 + e] = (T)(v + cst);
}

// The constants of the truncated kernels (Remark stokeslet_const_corr; the C^1 gauge of the
// D = 0 biharmonic kernel) times the total strength: ucst[j] = sum_a rconst[j][a] rho_sum[a].
// They are added to the potentials in FP64 at the leaf write-back rather than to the root grids,
// so that the FP32 expansions of the mixed path do not carry them (a constant has no gradient).
__global__ void k_root_const(int du, int drho, const double* __restrict__ rconst, const double* __restrict__ rho_sum,
                             double* __restrict__ ucst) {
    const int j = threadIdx.x;
    if (j >= du) return;
    double v = 0;
    for (int a = 0; a < drho; ++a) v += rconst[j * drho + a] * rho_sum[a];
    ucst[j] = v;
}

// Root proxies entering the structure factor of a non-exact tiling (Sec. 4.3): the cube's own
// proxy for a cube inside Omega (class 0), nothing for a padding cube (class 2); cut cubes
// (class 1) are filled afterwards from their original sources by k_anterp.
template <class T>
__global__ void k_chi_proxy(int Mtot, int drho, int p3, const int* __restrict__ cls, const T* __restrict__ proxy,
                            T* __restrict__ chip) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)Mtot * drho * p3) return;
    const int cube = (int)(t / ((int64_t)drho * p3));
    chip[t] = cls[cube] == 0 ? proxy[t] : T(0);
}

// ---- root far field as DFTs over the cube index (Sec. 3.4 "Case 1: elongated cuboid" and
// "Case 2: two long sides", Eqs. beta_def, 1d-DFT-beta, structfac-case1-wDFTCoeffs,
// ufar_inverse_fft; Sec. 5.4 for free directions, Eqs. kappaqdef, beta_hat_oversampled,
// structurefac_oversampled_fft) ------------------------------------------------------------
// On an exact tiling of M1 x M2 x M3 cubes of side s whose wavenumbers are k_a = 2 pi n_a /
// (Q_a s) on every axis (Q_a = M_a on a periodic axis, the oversampled length Q_a >= M_a on a
// free one), the phase of cube m is exp(-i k . c_0) prod_a exp(-2 pi i (n_a mod Q_a) m_a / Q_a).
// Forward: the partial sums beta_m(j3; k1, k2) (contracted over j1 and j2 per cube) are summed
// over m1 and m2 at the one frequency each (k1, k2) needs, then transformed over m3 to all Q3
// frequencies (zero padded from M3 to Q3); chi(k) contracts j3 of that transform at n3 mod Q3.
// Evaluation, the transpose: sums over the modes grouped by n3 mod Q3, an inverse transform of
// the groups to every m3, then per cube the k2 -> j2 and k1 -> j1 contractions with that cube's
// phases for m2 and m1.  The transforms are direct sums, one thread per output: their cost is
// M3 Q3 n1 n2 p per component, against M n1 n2 n3 p for the direct sums over the cubes.

// A[(m3 drho + a) E + e] = sum_{m1, m2} exp(-2 pi i (s1 m1 / Q1 + s2 m2 / Q2)) beta[(m drho + a) E + e]
// with E = n1 n2 p, e = (i1 n2 + i2) p + j3, s_a = n_a mod Q_a of i_a, m = m1 + M1 (m2 + M2 m3)
__global__ void k_rootdft_fold12(int M1, int M2, int M3, int drho, int p, RootTab rt,
                                 const Cx<double>* __restrict__ beta, Cx<double>* __restrict__ A) {
    const int n2 = rt.n2, E = rt.n1 * n2 * p;
    const int64_t per = (int64_t)drho * E;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)M3 * per) return;
    const int m3 = (int)(id / per);
    const int64_t t = id % per;
    const int e = (int)(t % E);
    const int i1 = e / (n2 * p), i2 = (e / p) % n2;
    const int s1 = (int)rt.nmod[0][i1], s2 = (int)rt.nmod[1][i2];
    Cx<double> v = {0, 0};
    for (int m2 = 0; m2 < M2; ++m2) {
        const Cx<double> w2 = rt.roots[1][(int)(((int64_t)s2 * m2) % rt.Q[1])];
        for (int m1 = 0; m1 < M1; ++m1) {
            const Cx<double> w = cmul(rt.roots[0][(int)(((int64_t)s1 * m1) % rt.Q[0])], w2);
            const int64_t m = m1 + (int64_t)M1 * (m2 + (int64_t)M2 * m3);
            cfma(v, cconj(w), beta[m * per + t]);
        }
    }
    A[id] = v;
}

// bhat[(s drho + a) E + e] = sum_{m3 < M3} exp(-2 pi i s m3 / Q3) A[(m3 drho + a) E + e], s < Q3
__global__ void k_rootdft_fwd3(int M3, int drho, int E, RootTab rt, const Cx<double>* __restrict__ A,
                               Cx<double>* __restrict__ bhat) {
    const int Q3 = rt.Q[2];
    const int64_t per = (int64_t)drho * E;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)Q3 * per) return;
    const int sidx = (int)(id / per);
    const int64_t t = id % per;
    Cx<double> v = {0, 0};
    for (int m = 0; m < M3; ++m) cfma(v, cconj(rt.roots[2][(int)(((int64_t)sidx * m) % Q3)]), A[(size_t)m * per + t]);
    bhat[id] = v;
}

// chi(k) for component a (all cubes as one): exp(-i k . c_0) sum_j3 S3(j3, k3) bhat_{n3 mod Q3}
__global__ void k_rootdft_chi(int drho, int p, Geo g, RootTab rt, const Cx<double>* __restrict__ bhat,
                              Cx<double>* __restrict__ chi) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)drho * rt.nmode) return;
    const int a = (int)(t / rt.nmode), e = (int)(t % rt.nmode);
    const int n2 = rt.n2, n3 = rt.n3, E = rt.n1 * n2 * p;
    const int i1 = e / (n2 * n3), i2 = (e / n3) % n2, i3 = e % n3;
    const int sm = (int)rt.nmod[2][i3];
    const Cx<double>* b = bhat + ((size_t)sm * drho + a) * E + ((size_t)i1 * n2 + i2) * p;
    Cx<double> v = {0, 0};
    for (int k = 0; k < p; ++k) cfma(v, rt.S[2][i3 * p + k], b[k]);
    const double h = 0.5 * g.s;
    const double ph = -(rt.kax[0][i1] + rt.kax[1][i2] + rt.kax[2][i3]) * h;
    double sn, cs;
    sincos(ph, &sn, &cs);
    chi[t] = cmul(v, Cx<double>{cs, sn});
}

// evaluation, k3 -> j3 grouped by s = n3 mod Q3: C2[(s du + j) E + e] =
//   sum_{i3 : n3 mod Q3 = s} conj(S3(j3, k3)) exp(i k . c_0) uhat_j(k)
__global__ void k_rootdft_bwd1(int du, int p, Geo g, RootTab rt, const Cx<double>* __restrict__ uhat,
                               Cx<double>* __restrict__ C2) {
    const int n2 = rt.n2, n3 = rt.n3, Q3 = rt.Q[2], per = rt.n1 * n2 * p;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)Q3 * du * per) return;
    const int job = (int)(id / per), e = (int)(id % per);
    const int sm = job / du, j = job % du;
    const int i12 = e / p, j3 = e % p;
    const int i1 = i12 / n2, i2 = i12 % n2;
    const double h = 0.5 * g.s;
    // consecutive indices i3 are consecutive n3: the group is every Q3-th index from its first
    const int first = ((sm - (int)rt.nmod[2][0]) % Q3 + Q3) % Q3;
    Cx<double> v = {0, 0};
    for (int i3 = first; i3 < n3; i3 += Q3) {
        if ((int)rt.nmod[2][i3] != sm) continue;
        const double ph = (rt.kax[0][i1] + rt.kax[1][i2] + rt.kax[2][i3]) * h;
        double sn, cs;
        sincos(ph, &sn, &cs);
        const Cx<double> gk = cmul(uhat[(size_t)j * rt.nmode + (size_t)i12 * n3 + i3], Cx<double>{cs, sn});
        cfma(v, cconj(rt.S[2][i3 * p + j3]), gk);
    }
    C2[id] = v;
}

// inverse transform to the cube index m3: Dm[(m3 du + j) E + e] = sum_{s < Q3} exp(2 pi i s m3 / Q3)
//   C2[(s du + j) E + e]
__global__ void k_rootdft_idft3(int M3, int du, int E, RootTab rt, const Cx<double>* __restrict__ C2,
                                Cx<double>* __restrict__ Dm) {
    const int Q3 = rt.Q[2];
    const int64_t per = (int64_t)du * E;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)M3 * per) return;
    const int m3 = (int)(id / per);
    const int64_t t = id % per;
    Cx<double> v = {0, 0};
    for (int sidx = 0; sidx < Q3; ++sidx)
        cfma(v, rt.roots[2][(int)(((int64_t)sidx * m3) % Q3)], C2[(size_t)sidx * per + t]);
    Dm[id] = v;
}

// per cube m = m1 + M1 (m2 + M2 m3), k2 -> j2 with the cube's phase for m2:
//   C1[(m du + j) n1 p^2 + (i1 p + j2) p + j3] =
//     sum_i2 conj(S2(j2, k2)) exp(2 pi i s2 m2 / Q2) Dm[(m3 du + j) E + (i1 n2 + i2) p + j3]
__global__ void k_rootdft_bwd2(int Mtot, int du, int p, Geo g, RootTab rt, const Cx<double>* __restrict__ Dm,
                               Cx<double>* __restrict__ C1) {
    const int p2 = p * p, n2 = rt.n2, per = rt.n1 * p2, E = rt.n1 * n2 * p;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)Mtot * du * per) return;
    const int job = (int)(id / per), e = (int)(id % per);
    const int m = job / du, j = job % du;
    const int m2 = (m / g.M[0]) % g.M[1], m3 = m / (g.M[0] * g.M[1]);
    const int i1 = e / p2, j2 = (e / p) % p, j3 = e % p;
    const Cx<double>* c = Dm + ((size_t)m3 * du + j) * E + (size_t)i1 * n2 * p + j3;
    Cx<double> v = {0, 0};
    for (int k = 0; k < n2; ++k) {
        const Cx<double> w = rt.roots[1][(int)(((int64_t)rt.nmod[1][k] * m2) % rt.Q[1])];
        cfma(v, cmul(cconj(rt.S[1][k * p + j2]), w), c[(size_t)k * p]);
    }
    C1[id] = v;
}

// per cube, k1 -> j1 with the cube's phase for m1, real part: local[(m du + j) p^3 + e]
// (= or += with add: a second root part adds to the first)
template <class T>
__global__ void k_rootdft_bwd3(int Mtot, int du, int p, Geo g, RootTab rt, const Cx<double>* __restrict__ C1,
                               T* __restrict__ local, int add) {
    const int p2 = p * p, p3 = p2 * p;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= (int64_t)Mtot * du * p3) return;
    const int job = (int)(id / p3), e = (int)(id % p3);
    const int m1 = (job / du) % g.M[0];
    const int j1 = e / p2, r = e % p2;
    const Cx<double>* c = C1 + (size_t)job * rt.n1 * p2 + r;
    double v = 0;
    for (int k = 0; k < rt.n1; ++k) {
        const Cx<double> w = rt.roots[0][(int)(((int64_t)rt.nmod[0][k] * m1) % rt.Q[0])];
        const Cx<double> f = cmul(cconj(rt.S[0][k * p + j1]), w);
        const Cx<double> b = c[(size_t)k * p2];
        v += f.x * b.x - f.y * b.y;
    }
    const size_t o = (size_t)job * p3 + e;
    local[o] = add ? (T)((double)local[o] + v) : (T)v;
}

// Position part of the vector-Jacobian product (reverse-mode derivative of the sums for a
// kernel with K(-x) = K(x)^T): d[a][i] = sum_j gu[a][i][j] g[a][j] + sum_l gv[a][i][l] rho[a][l],
// gu the field gradient of the forward sum, gv that of the sum with strengths g (d_u = d_rho).
__global__ void k_vjp_points(int64_t N, int du, const double* __restrict__ gu, const double* __restrict__ g,
                             const double* __restrict__ gv, const double* __restrict__ rho, double* __restrict__ d) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 3 * N) return;
    const int64_t a = t / 3;
    const int i = (int)(t - 3 * a);
    double v = 0;
    for (int j = 0; j < du; ++j)
        v = fma(gu[(a * 3 + i) * du + j], g[a * du + j], fma(gv[(a * 3 + i) * du + j], rho[a * du + j], v));
    d[t] = v;
}

// The stresslet's vector-Jacobian product.  The periodized stresslet T_jlm is fully symmetric in
// (j, l, m) and odd in x, so dL/dQ_s,lm = sum_t g_t,j T_jlm(x_t - x_s) = -S[g (x) e_m]_l(x_s),
// S[Q] the stresslet sum with strengths Q: three evaluations with the strengths g (x) e_m.
// k_vjp_stresslet_q forms those strengths (component m of q), k_vjp_stresslet_acc accumulates
// dL/dQ[s][l][m] = -u_m[s][l] and the source part of dL/dx_s, -sum_lm Q_s,lm d_i S[g (x) e_m]_l.
__global__ void k_vjp_stresslet_q(int64_t N, int m, const double* __restrict__ g, double* __restrict__ q) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 9 * N) return;
    const int64_t s = t / 9;
    const int e = (int)(t - 9 * s), j = e / 3, k = e - 3 * j;
    q[t] = (k == m) ? g[s * 3 + j] : 0.0;
}

__global__ void k_vjp_stresslet_acc(int64_t N, int m, const double* __restrict__ um, const double* __restrict__ gm,
                                    const double* __restrict__ Q, double* __restrict__ dQ,
                                    double* __restrict__ dx) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    if (dQ)
        for (int l = 0; l < 3; ++l) dQ[s * 9 + l * 3 + m] = -um[s * 3 + l];
    if (dx)
        for (int i = 0; i < 3; ++i) {
            double v = dx[s * 3 + i];
            for (int l = 0; l < 3; ++l) v = fma(-Q[s * 9 + l * 3 + m], gm[(s * 3 + i) * 3 + l], v);
            dx[s * 3 + i] = v;
        }
}

// target part of dL/dx for a kernel that is not self-adjoint: d[a][i] = sum_j gu[a][i][j] g[a][j]
__global__ void k_vjp_target(int64_t N, int du, const double* __restrict__ gu, const double* __restrict__ g,
                             double* __restrict__ d) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 3 * N) return;
    const int64_t a = t / 3;
    const int i = (int)(t - 3 * a);
    double v = 0;
    for (int j = 0; j < du; ++j) v = fma(gu[(a * 3 + i) * du + j], g[a * du + j], v);
    d[t] = v;
}

// ------------------------------------------------------------------------------------------
// Residual kernels K_R(x; nu) (App. B, Remark scaling_stokes_split) and their gradients for one
// source-target pair; the 1/(4 pi) or 1/(8 pi) factor is applied once per target.  q, f, g are
// Chebyshev series in t = 2 r^2/nu^2 - 1 for (int_0^rho phi)/rho, phi(rho), phi'(rho)/rho.
template <class T, int K, bool GRAD>
struct Pair;

template <class T, bool GRAD>
struct Pair<T, DMK_LAPLACE, GRAD> {
    static constexpr int DR = 1, DU = 1;
    template <class SE>
    __device__ __forceinline__ static void eval(const SE& se, T dx, T dy, T dz, T r2, T inv_nu, const T* rho, T* u,
                                                T* gr) {
        const T rinv = rsqrt_t(r2);
        const T q = se(kSerQ);
        u[0] = fma(rho[0], rinv - T(2) * inv_nu * q, u[0]);
        if (GRAD) {
            const T f = se(kSerF);
            const T ri2 = rinv * rinv;
            const T gfac = rho[0] * (ri2 * rinv + T(2) * inv_nu * (f - q) * ri2);
            gr[0] = fma(-dx, gfac, gr[0]);
            gr[1] = fma(-dy, gfac, gr[1]);
            gr[2] = fma(-dz, gfac, gr[2]);
        }
    }
    __device__ __forceinline__ static float rsqrt_t(float v) { return rsqrtf(v); }
    __device__ __forceinline__ static double rsqrt_t(double v) { return rsqrt(v); }
};

template <class T>
__device__ __forceinline__ T rsqrt_any(T v);
template <> __device__ __forceinline__ float rsqrt_any<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_any<double>(double v) { return rsqrt(v); }

template <class T, bool GRAD>
struct Pair<T, DMK_STOKESLET, GRAD> {
    static constexpr int DR = 3, DU = 3;
    template <class SE>
    __device__ __forceinline__ static void eval(const SE& se, T dx, T dy, T dz, T r2, T inv_nu, const T* rho, T* u,
                                                T* gr) {
        const T rinv = rsqrt_any(r2), ri2 = rinv * rinv;
        const T q = se(kSerQ);
        const T f = se(kSerF);
        const T A = rinv - T(2) * inv_nu * (q + f);
        const T Bc = ri2 * rinv - T(2) * inv_nu * (q - f) * ri2;
        const T x[3] = {dx, dy, dz};
        const T xr = dx * rho[0] + dy * rho[1] + dz * rho[2];
        for (int j = 0; j < 3; ++j) u[j] += A * rho[j] + Bc * xr * x[j];
        if (GRAD) {
            const T dq = se(kSerDQ);
            const T df = se(kSerDF);
            const T r = r2 * rinv;
            const T dsdr = T(2) * r * inv_nu * inv_nu;
            const T Ap = -ri2 - T(2) * inv_nu * (dq + df) * dsdr;
            const T Bp = T(-3) * ri2 * ri2 - T(2) * inv_nu * ((dq - df) * dsdr * ri2 - T(2) * (q - f) * ri2 * rinv);
            for (int i = 0; i < 3; ++i) {
                const T xi_r = x[i] * rinv;
                for (int j = 0; j < 3; ++j)
                    gr[i * 3 + j] += Ap * xi_r * rho[j] + Bp * xi_r * xr * x[j]
                                     + Bc * (rho[i] * x[j] + (i == j ? xr : T(0)));
            }
        }
    }
};

template <class T, bool GRAD>
struct Pair<T, DMK_STRESSLET, GRAD> {
    static constexpr int DR = 9, DU = 3;
    // u_j = Pd v_j/(8 pi) - (3/(4 pi)) Po x_j w, v = Qx + Q^T x + x tr Q, w = x^T Q x,
    // Pd = T_diag/r^3 = -2 g/nu^3, Po = T_offd/r^5.  Stored as 8 pi * u: Pd v_j - 6 Po x_j w.
    template <class SE>
    __device__ __forceinline__ static void eval(const SE& se, T dx, T dy, T dz, T r2, T inv_nu, const T* Q, T* u,
                                                T* gr) {
        const T rinv = rsqrt_any(r2), ri2 = rinv * rinv;
        const T q = se(kSerQ);
        const T f = se(kSerF);
        const T g = se(kSerG);
        const T in3 = inv_nu * inv_nu * inv_nu;
        const T Pd = T(-2) * g * in3;
        const T Po = ri2 * ri2 * rinv - T(2) * inv_nu * (q - f) * ri2 * ri2 - T(2.0 / 3.0) * g * in3 * ri2;
        const T x[3] = {dx, dy, dz};
        T Qx[3], QTx[3];
        for (int j = 0; j < 3; ++j) {
            Qx[j] = Q[j * 3] * x[0] + Q[j * 3 + 1] * x[1] + Q[j * 3 + 2] * x[2];
            QTx[j] = Q[j] * x[0] + Q[3 + j] * x[1] + Q[6 + j] * x[2];
        }
        const T tr = Q[0] + Q[4] + Q[8];
        const T w = x[0] * Qx[0] + x[1] * Qx[1] + x[2] * Qx[2];
        T v[3];
        for (int j = 0; j < 3; ++j) {
            v[j] = Qx[j] + QTx[j] + x[j] * tr;
            u[j] += Pd * v[j] - T(6) * Po * x[j] * w;
        }
        if (GRAD) {
            const T dq = se(kSerDQ);
            const T df = se(kSerDF);
            const T dg = se(kSerDG);
            const T r = r2 * rinv;
            const T dsdr = T(2) * r * inv_nu * inv_nu;
            const T Pdp = T(-2) * dg * dsdr * in3;
            const T Pop = T(-5) * ri2 * ri2 * ri2
                          - T(2) * inv_nu * ((dq - df) * dsdr * ri2 * ri2 - T(4) * (q - f) * ri2 * ri2 * rinv)
                          - T(2.0 / 3.0) * in3 * (dg * dsdr * ri2 - T(2) * g * ri2 * rinv);
            for (int i = 0; i < 3; ++i) {
                const T xi_r = x[i] * rinv;
                const T dw = Qx[i] + QTx[i];
                for (int j = 0; j < 3; ++j) {
                    const T dv = Q[j * 3 + i] + Q[i * 3 + j] + (i == j ? tr : T(0));
                    gr[i * 3 + j] += Pdp * xi_r * v[j] + Pd * dv
                                     - T(6) * (Pop * xi_r * x[j] * w + Po * ((i == j ? w : T(0)) + x[j] * dw));
                }
            }
        }
    }
};

template <class T, bool GRAD>
struct Pair<T, DMK_ROTLET, GRAD> {
    static constexpr int DR = 3, DU = 3;
    // u = (tau x x) Oc/(8 pi), Oc = Omega_offd / r^3
    template <class SE>
    __device__ __forceinline__ static void eval(const SE& se, T dx, T dy, T dz, T r2, T inv_nu, const T* tau, T* u,
                                                T* gr) {
        const T rinv = rsqrt_any(r2), ri2 = rinv * rinv;
        const T q = se(kSerQ);
        const T f = se(kSerF);
        const T Oc = ri2 * rinv - T(2) * inv_nu * (q - f) * ri2;
        const T x[3] = {dx, dy, dz};
        const T c[3] = {tau[1] * dz - tau[2] * dy, tau[2] * dx - tau[0] * dz, tau[0] * dy - tau[1] * dx};
        for (int j = 0; j < 3; ++j) u[j] += Oc * c[j];
        if (GRAD) {
            const T dq = se(kSerDQ);
            const T df = se(kSerDF);
            const T r = r2 * rinv;
            const T dsdr = T(2) * r * inv_nu * inv_nu;
            const T Op = T(-3) * ri2 * ri2 - T(2) * inv_nu * ((dq - df) * dsdr * ri2 - T(2) * (q - f) * ri2 * rinv);
            for (int i = 0; i < 3; ++i) {
                const T xi_r = x[i] * rinv;
                for (int j = 0; j < 3; ++j) {
                    // d_i (tau x x)_j = eps_jli tau_l
                    T dc = 0;
                    const int l = 3 - i - j;
                    if (i != j) dc = (((j + 1) % 3) == l ? T(1) : T(-1)) * tau[l];
                    gr[i * 3 + j] += Op * xi_r * c[j] + Oc * dc;
                }
            }
        }
    }
};

template <int K> struct KScale { static constexpr double v = (K == DMK_LAPLACE) ? 0.07957747154594767 : 0.039788735772973836; };

// ------------------------------------------------------------------------------------------
// Outputs and per-point inputs of the leaf stage (Sec. 3.1.5, Sec. 2.4): potentials and
// gradients in input order, the sort permutation, strengths, self terms, FP32 point records.
struct LeafOut {
    double* pot;
    double* grad;      // may be null
    const int* perm;   // sorted point -> input point (images of a non-exact tiling: >= n_orig)
    const int* orig;   // sorted point -> the original point it is (or is an image of)
    int64_t n_orig;    // points with outputs: perm < n_orig
    const double* rs;  // sorted strengths (FP64)
    const double* self_val;   // du x drho at nu = 1
    const double* self_grad;  // 3 x du x drho at nu = 1
    const float4* pk;         // FP32 path: one record per sorted point (point_record layout)
    const double* ucst;       // du constants added to every potential (truncated-kernel gauge
                              // constants times the total strength), or null
};


}  // namespace dmk
