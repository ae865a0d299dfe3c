// Register-blocked tensor contractions for the upward pass and the shift to children, and the
// leaf stage with in-support pair compaction.  These replace the generic versions in
// dmk_kernels.cuh when p <= kMaxPFast.
//
// A p x p x p tensor sits in shared memory x-major with an odd row pitch P = p | 1, so that
// p-long fibers along any axis, one per thread, are read without bank conflicts.  Contracting
// one axis with a p x p operator is then "each thread owns one fiber": it reads its p inputs
// and accumulates p outputs in registers, with the operator rows loaded as shared-memory
// broadcasts.  Operator rows are zero-padded to MAXP so the unrolled loops need no guards.
#pragma once
#include "dmk_kernels.cuh"

namespace dmk {

constexpr int kMaxPFast = 24;

__host__ __device__ __forceinline__ int odd_pitch(int p) { return p | 1; }

// element (i0, i1, i2) of a padded tensor
__device__ __forceinline__ int pidx(int i0, int i1, int i2, int p, int P) { return (i0 * p + i1) * P + i2; }

// out[j] = sum_k M[k][j] * in(fiber, k) for the fiber (fa, fb) across axis ax
template <class T, int MAXP>
__device__ __forceinline__ void fiber_contract(const T* in, int p, int P, int ax, int fa, int fb, const T* M,
                                               T (&acc)[MAXP]) {
#pragma unroll
    for (int j = 0; j < MAXP; ++j) acc[j] = 0;
    for (int k = 0; k < p; ++k) {
        const int e = (ax == 2) ? pidx(fa, fb, k, p, P) : (ax == 1) ? pidx(fa, k, fb, p, P) : pidx(k, fa, fb, p, P);
        const T x = in[e];
        const T* row = M + k * MAXP;
#pragma unroll
        for (int j = 0; j < MAXP; ++j) acc[j] = fma(row[j], x, acc[j]);
    }
}

// acc[j] += sum_k M[k][j] * in(fiber, k)
template <class T, int MAXP>
__device__ __forceinline__ void fiber_accum(const T* in, int p, int P, int ax, int fa, int fb, const T* M,
                                            T (&acc)[MAXP]) {
    for (int k = 0; k < p; ++k) {
        const int e = (ax == 2) ? pidx(fa, fb, k, p, P) : (ax == 1) ? pidx(fa, k, fb, p, P) : pidx(k, fa, fb, p, P);
        const T x = in[e];
        const T* row = M + k * MAXP;
#pragma unroll
        for (int j = 0; j < MAXP; ++j) acc[j] = fma(row[j], x, acc[j]);
    }
}

template <class T, int MAXP>
__device__ __forceinline__ void fiber_store(T* out, int p, int P, int ax, int fa, int fb, const T (&acc)[MAXP]) {
#pragma unroll
    for (int j = 0; j < MAXP; ++j) {
        if (j < p) {
            const int e = (ax == 2) ? pidx(fa, fb, j, p, P) : (ax == 1) ? pidx(fa, j, fb, p, P) : pidx(j, fa, fb, p, P);
            out[e] = acc[j];
        }
    }
}

// operator rows into shared memory: Ms[k * MAXP + j] = src(k, j) (zero beyond p)
template <class T, int MAXP, class F>
__device__ __forceinline__ void load_op(T* Ms, int p, F src) {
    for (int e = threadIdx.x; e < MAXP * MAXP; e += blockDim.x) {
        const int k = e / MAXP, j = e % MAXP;
        Ms[e] = (k < p && j < p) ? src(k, j) : T(0);
    }
}

template <class T>
__device__ __forceinline__ void load_padded(T* dst, const T* src, int p, int P) {
    const int p3 = p * p * p;
    for (int e = threadIdx.x; e < p3; e += blockDim.x) dst[(e / p) * P + (e % p)] = src[e];
}

// Upward pass child -> parent (Sec. 3.1.2): parent = sum_o (I_o^T x I_o^T x I_o^T) child_o.
// Thread f < p^2 owns the x-fiber (i1, i2) of the parent across all eight children.
template <class T, int MAXP>
__global__ void __launch_bounds__(576) k_upward2(int n, const int* __restrict__ nl_box, BoxArrays B, Tab<T> tab,
                                                 T* __restrict__ proxy) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, P = odd_pitch(p), drho = tab.d_rho;
    T* Mo = reinterpret_cast<T*>(dsmem);                 // 2 x MAXP x MAXP
    T* bufA = Mo + 2 * MAXP * MAXP;
    T* bufB = bufA + p * p * P;
    // rows k = child node, columns = parent index: I[o][k][c]
    for (int o = 0; o < 2; ++o)
        load_op<T, MAXP>(Mo + o * MAXP * MAXP, p, [&](int k, int j) { return tab.Ioct[(o * p + k) * p + j]; });
    const int f = threadIdx.x;
    const bool own = f < p2;
    const int fa = own ? f / p : 0, fb = own ? f % p : 0;
    for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const int Pb = nl_box[bi];
        const int c0 = B.child0[Pb];
        for (int a = 0; a < drho; ++a) {
            T acc[MAXP];
#pragma unroll
            for (int j = 0; j < MAXP; ++j) acc[j] = 0;
            for (int o = 0; o < 8; ++o) {
                __syncthreads();
                load_padded(bufA, proxy + ((size_t)(c0 + o) * drho + a) * p3, p, P);
                __syncthreads();
                T t[MAXP];
                if (own) {
                    fiber_contract<T, MAXP>(bufA, p, P, 2, fa, fb, Mo + ((o >> 2) & 1) * MAXP * MAXP, t);
                    fiber_store<T, MAXP>(bufB, p, P, 2, fa, fb, t);
                }
                __syncthreads();
                if (own) {
                    fiber_contract<T, MAXP>(bufB, p, P, 1, fa, fb, Mo + ((o >> 1) & 1) * MAXP * MAXP, t);
                    fiber_store<T, MAXP>(bufA, p, P, 1, fa, fb, t);
                }
                __syncthreads();
                if (own) fiber_accum<T, MAXP>(bufA, p, P, 0, fa, fb, Mo + (o & 1) * MAXP * MAXP, acc);
            }
            if (own) {
                T* out = proxy + ((size_t)Pb * drho + a) * p3;
#pragma unroll
                for (int j = 0; j < MAXP; ++j)
                    if (j < p) out[(j * p + fa) * p + fb] = acc[j];
            }
        }
    }
}

// Shift to children (Sec. 3.1.4).  Non-leaf child: local += (I_o x I_o x I_o) parent.  Leaf child:
// local += (A_o x A_o x A_o) parent, A_o = C I_o, i.e. the Chebyshev coefficients of the child's
// interpolant, which is what the leaf stage evaluates.
template <class T, int MAXP>
__global__ void __launch_bounds__(576) k_shift2(int n, const int* __restrict__ nl_box, BoxArrays B, Tab<T> tab,
                                                T* __restrict__ local) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, P = odd_pitch(p), du = tab.d_u;
    T* MI = reinterpret_cast<T*>(dsmem);                 // 2 x MAXP x MAXP, rows k = parent index
    T* MA = MI + 2 * MAXP * MAXP;
    T* bufP = MA + 2 * MAXP * MAXP;
    T* t1 = bufP + p * p * P;
    T* t2 = t1 + p * p * P;
    for (int o = 0; o < 2; ++o) {
        load_op<T, MAXP>(MI + o * MAXP * MAXP, p, [&](int k, int j) { return tab.Ioct[(o * p + j) * p + k]; });
        load_op<T, MAXP>(MA + o * MAXP * MAXP, p, [&](int k, int j) { return tab.Aoct[(o * p + j) * p + k]; });
    }
    const int f = threadIdx.x;
    const bool own = f < p2;
    const int fa = own ? f / p : 0, fb = own ? f % p : 0;
    for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const int Pb = nl_box[bi];
        const int c0 = B.child0[Pb];
        for (int j = 0; j < du; ++j) {
            __syncthreads();
            load_padded(bufP, local + ((size_t)Pb * du + j) * p3, p, P);
            for (int o = 0; o < 8; ++o) {
                const int C = c0 + o;
                const T* Mbase = (B.child0[C] < 0) ? MA : MI;
                __syncthreads();
                T t[MAXP];
                if (own) {
                    fiber_contract<T, MAXP>(bufP, p, P, 2, fa, fb, Mbase + ((o >> 2) & 1) * MAXP * MAXP, t);
                    fiber_store<T, MAXP>(t1, p, P, 2, fa, fb, t);
                }
                __syncthreads();
                if (own) {
                    fiber_contract<T, MAXP>(t1, p, P, 1, fa, fb, Mbase + ((o >> 1) & 1) * MAXP * MAXP, t);
                    fiber_store<T, MAXP>(t2, p, P, 1, fa, fb, t);
                }
                __syncthreads();
                if (own) {
                    fiber_contract<T, MAXP>(t2, p, P, 0, fa, fb, Mbase + (o & 1) * MAXP * MAXP, t);
                    T* out = local + ((size_t)C * du + j) * p3;
#pragma unroll
                    for (int jj = 0; jj < MAXP; ++jj)
                        if (jj < p) out[(jj * p + fa) * p + fb] += t[jj];
                }
            }
        }
    }
}

// Grid values -> Chebyshev coefficients in place, for leaves whose grid did not come through
// k_shift2 (root-level leaves, and every leaf when p > kMaxPFast).
template <class T>
__global__ void k_grid2coef(int n, const int* __restrict__ boxes, const int* __restrict__ level, int root_only,
                            Tab<T> tab, T* __restrict__ local, unsigned char* scratch, size_t per_cta, int use_smem) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, du = tab.d_u;
    T* t1 = reinterpret_cast<T*>(work_base(scratch, per_cta, use_smem));
    T* t2 = t1 + p3;
    for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const int box = boxes[bi];
        if (root_only && level[box] != 0) continue;
        for (int j = 0; j < du; ++j) {
            T* u = local + ((size_t)box * du + j) * p3;
            __syncthreads();
            for (int e = threadIdx.x; e < p3; e += blockDim.x) {
                const int i12 = e / p, n3 = e % p;
                T v = 0;
                for (int k = 0; k < p; ++k) v = fma(tab.Cm[n3 * p + k], u[i12 * p + k], v);
                t1[e] = v;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < p3; e += blockDim.x) {
                const int i1 = e / p2, n2 = (e / p) % p, n3 = e % p;
                T v = 0;
                for (int k = 0; k < p; ++k) v = fma(tab.Cm[n2 * p + k], t1[(i1 * p + k) * p + n3], v);
                t2[e] = v;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < p3; e += blockDim.x) {
                const int n1 = e / p2, rr = e % p2;
                T v = 0;
                for (int k = 0; k < p; ++k) v = fma(tab.Cm[n1 * p + k], t2[k * p2 + rr], v);
                u[e] = v;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Leaf stage (Sec. 3.1.5, Sec. 2.4), local[leaf] holding Chebyshev coefficients.
// (2) expansion and gradient at the targets: warp per target, lane = n3, coefficients read
//     through L1; (3) residual sums: the sources of all direct-list entries stream through
//     shared memory in chunks of kSrcChunk; each thread (one target) first collects the
//     in-support sources of the chunk into a byte queue, then evaluates only those, so the
//     out-of-support majority costs a distance test and nothing more; (4) self correction and
//     the FP64 write-back in input order.
constexpr int kLeaf2Threads = 128;
constexpr int kSrcChunk = 256;

template <class T, int K, bool GRAD>
__global__ void __launch_bounds__(kLeaf2Threads) k_leaf2(int nleaf, const int* __restrict__ leaves, BoxArrays B,
                                                        Tab<T> tab, Geo g, const T* __restrict__ coef,
                                                        const double* __restrict__ xs, int64_t N,
                                                        const int* __restrict__ doffs,
                                                        const DirectEntry* __restrict__ dl, LeafOut out) {
    using Pr = Pair<T, K, GRAD>;
    constexpr int DR = Pr::DR, DU = Pr::DU, NR = DU * 4;
    const int p = tab.p, p2 = p * p, p3 = p2 * p;
    __shared__ double res[kLeaf2Threads][NR];
    // FP32 path: coordinates relative to the leaf centre as hi + lo pairs, so that the
    // difference of two nearby points keeps full relative precision (hi - hi is exact by
    // Sterbenz when the points are close; lo - lo adds the remainder)
    constexpr bool kTwo = sizeof(T) == 4;
    constexpr int kLo = kTwo ? kSrcChunk : 1;
    __shared__ T sx[kSrcChunk], sy[kSrcChunk], sz[kSrcChunk], sinv[kSrcChunk], snu2[kSrcChunk];
    __shared__ T sxl[kLo], syl[kLo], szl[kLo];
    __shared__ T tv[kLeaf2Threads / 32][4][64];
    // dynamic: the in-support queue (source slot per (position, thread)) and staged strengths
    unsigned char (*q)[kLeaf2Threads] = reinterpret_cast<unsigned char (*)[kLeaf2Threads]>(dsmem);
    T (*sr)[DR] = reinterpret_cast<T (*)[DR]>(dsmem + kSrcChunk * kLeaf2Threads);
    __shared__ T fits[256];
    for (int e = threadIdx.x; e < min(256, tab.n_q + tab.n_f + tab.n_g + tab.n_dq + tab.n_df + tab.n_dg);
         e += blockDim.x)
        fits[e] = tab.fit[e];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const int box = leaves[li];
        const int l = B.level[box];
        const double r = g.s / (double)(1 << l), half = 0.5 * r;
        const double c[3] = {(B.ix[3 * box] + 0.5) * r, (B.ix[3 * box + 1] + 0.5) * r, (B.ix[3 * box + 2] + 0.5) * r};
        const int st = B.start[box], en = B.end[box];
        for (int t0 = st; t0 < en; t0 += kLeaf2Threads) {
            const int nt = min(kLeaf2Threads, en - t0);
            __syncthreads();
            // (2) Chebyshev evaluation, warp per target
            for (int tt = warp; tt < nt; tt += nwarp) {
                const int tg = t0 + tt;
                T xi[3];
                for (int a = 0; a < 3; ++a) {
                    T v = (T)((xs[a * N + tg] - c[a]) / half);
                    xi[a] = v > T(1) ? T(1) : (v < T(-1) ? T(-1) : v);
                }
                // T_n and T_n' = n U_{n-1}: x and y in shared memory (lane 0 writes), z in registers
                T Tz0 = 0, Tz1 = 0, dTz0 = 0, dTz1 = 0;
                {
                    T Tm1[3], Tm2[3], Um1[3], Um2[3];
                    for (int n = 0; n < p; ++n) {
                        T Tn[3], dTn[3];
                        for (int a = 0; a < 3; ++a) {
                            if (n == 0) {
                                Tn[a] = 1; dTn[a] = 0;
                                Tm1[a] = 1; Tm2[a] = 0; Um1[a] = 1; Um2[a] = 0;
                            } else if (n == 1) {
                                Tn[a] = xi[a]; dTn[a] = 1;
                                Tm2[a] = Tm1[a]; Tm1[a] = xi[a];
                                Um2[a] = Um1[a]; Um1[a] = 2 * xi[a];
                            } else {
                                Tn[a] = 2 * xi[a] * Tm1[a] - Tm2[a];
                                dTn[a] = (T)n * Um1[a];
                                const T Un = 2 * xi[a] * Um1[a] - Um2[a];
                                Tm2[a] = Tm1[a]; Tm1[a] = Tn[a];
                                Um2[a] = Um1[a]; Um1[a] = Un;
                            }
                        }
                        if (lane == (n & 31)) {
                            if (n < 32) { Tz0 = Tn[2]; dTz0 = dTn[2]; } else { Tz1 = Tn[2]; dTz1 = dTn[2]; }
                        }
                        if (lane == 0) {
                            tv[warp][0][n] = Tn[0]; tv[warp][1][n] = dTn[0];
                            tv[warp][2][n] = Tn[1]; tv[warp][3][n] = dTn[1];
                        }
                    }
                }
                __syncwarp();
                for (int j = 0; j < DU; ++j) {
                    const T* cj = coef + ((size_t)box * DU + j) * p3;
                    T S[2] = {0, 0}, Sx[2] = {0, 0}, Sy[2] = {0, 0};
                    for (int h = 0; h < 2; ++h) {
                        const int n3 = lane + 32 * h;
                        if (n3 >= p) continue;
                        for (int n1 = 0; n1 < p; ++n1) {
                            T a0 = 0, a1 = 0;
                            const T* row = cj + (size_t)n1 * p2 + n3;
                            for (int n2 = 0; n2 < p; ++n2) {
                                const T cv = __ldg(row + n2 * p);
                                a0 = fma(tv[warp][2][n2], cv, a0);
                                a1 = fma(tv[warp][3][n2], cv, a1);
                            }
                            S[h] = fma(tv[warp][0][n1], a0, S[h]);
                            Sx[h] = fma(tv[warp][1][n1], a0, Sx[h]);
                            Sy[h] = fma(tv[warp][0][n1], a1, Sy[h]);
                        }
                    }
                    T v = S[0] * Tz0 + S[1] * Tz1;
                    T gx = Sx[0] * Tz0 + Sx[1] * Tz1;
                    T gy = Sy[0] * Tz0 + Sy[1] * Tz1;
                    T gz = S[0] * dTz0 + S[1] * dTz1;
                    for (int o = 16; o > 0; o >>= 1) {
                        v += __shfl_xor_sync(0xffffffffu, v, o);
                        gx += __shfl_xor_sync(0xffffffffu, gx, o);
                        gy += __shfl_xor_sync(0xffffffffu, gy, o);
                        gz += __shfl_xor_sync(0xffffffffu, gz, o);
                    }
                    if (lane == 0) {
                        const double sc = 1.0 / half;
                        res[tt][j] = (double)v;
                        res[tt][DU + 0 * DU + j] = (double)gx * sc;
                        res[tt][DU + 1 * DU + j] = (double)gy * sc;
                        res[tt][DU + 2 * DU + j] = (double)gz * sc;
                    }
                }
                __syncwarp();
            }
            // (3) residual sums with in-support compaction
            const int tt = threadIdx.x;
            const bool act = tt < nt;
            T xt[3] = {0, 0, 0}, xtl[3] = {0, 0, 0};
            if (act)
                for (int a = 0; a < 3; ++a) {
                    const double v = xs[a * N + t0 + tt] - c[a];
                    xt[a] = (T)v;
                    if (kTwo) xtl[a] = (T)(v - (double)xt[a]);
                }
            // FP32 partial sums per chunk, folded into FP64 totals
            double accd[DU], gaccd[3 * DU];
            for (int j = 0; j < DU; ++j) accd[j] = 0;
            for (int j = 0; j < 3 * DU; ++j) gaccd[j] = 0;
            int e = doffs[li];
            const int e1 = doffs[li + 1];
            int eo = 0;
            while (e < e1) {
                __syncthreads();
                int filled = 0;
                while (filled < kSrcChunk && e < e1) {
                    const DirectEntry de = dl[e];
                    const int take = min(de.end - de.start - eo, kSrcChunk - filled);
                    const int lev = de.code >> 6;
                    const double sh0 = (double)(((de.code) & 3) - 1) * g.L[0];
                    const double sh1 = (double)(((de.code >> 2) & 3) - 1) * g.L[1];
                    const double sh2 = (double)(((de.code >> 4) & 3) - 1) * g.L[2];
                    const double inv = (double)(1 << lev) / g.s;
                    for (int k = threadIdx.x; k < take; k += blockDim.x) {
                        const int si = de.start + eo + k, slot = filled + k;
                        const double vx = xs[si] + sh0 - c[0], vy = xs[N + si] + sh1 - c[1],
                                     vz = xs[2 * N + si] + sh2 - c[2];
                        sx[slot] = (T)vx;
                        sy[slot] = (T)vy;
                        sz[slot] = (T)vz;
                        if (kTwo) {
                            sxl[slot] = (T)(vx - (double)sx[slot]);
                            syl[slot] = (T)(vy - (double)sy[slot]);
                            szl[slot] = (T)(vz - (double)sz[slot]);
                        }
                        sinv[slot] = (T)inv;
                        snu2[slot] = (T)(1.0 / (inv * inv));
                        for (int a = 0; a < DR; ++a) sr[slot][a] = (T)out.rs[(int64_t)si * DR + a];
                    }
                    filled += take;
                    eo += take;
                    if (eo == de.end - de.start) { ++e; eo = 0; }
                }
                __syncthreads();
                if (act) {
                    int cnt = 0;
                    for (int k = 0; k < filled; ++k) {
                        T dx = xt[0] - sx[k], dy = xt[1] - sy[k], dz = xt[2] - sz[k];
                        if (kTwo) {
                            dx += xtl[0] - sxl[k];
                            dy += xtl[1] - syl[k];
                            dz += xtl[2] - szl[k];
                        }
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < snu2[k] && r2 > T(0)) q[cnt++][tt] = (unsigned char)k;
                    }
                    T acc[DU], gacc[3 * DU];
                    for (int j = 0; j < DU; ++j) acc[j] = 0;
                    for (int j = 0; j < 3 * DU; ++j) gacc[j] = 0;
                    for (int i = 0; i < cnt; ++i) {
                        const int k = q[i][tt];
                        T dx = xt[0] - sx[k], dy = xt[1] - sy[k], dz = xt[2] - sz[k];
                        if (kTwo) {
                            dx += xtl[0] - sxl[k];
                            dy += xtl[1] - syl[k];
                            dz += xtl[2] - szl[k];
                        }
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        Pr::eval(tab, K == DMK_LAPLACE ? fits + tab.off_q : fits,
                                 K == DMK_LAPLACE ? fits + tab.off_f : fits, dx, dy, dz, r2, sinv[k], sr[k], acc,
                                 gacc);
                    }
                    for (int j = 0; j < DU; ++j) accd[j] += (double)acc[j];
                    for (int j = 0; j < 3 * DU; ++j) gaccd[j] += (double)gacc[j];
                }
            }
            __syncthreads();
            // (4) self correction and write-back (FP64)
            if (act) {
                const int tg = t0 + tt;
                const int oi = out.perm[tg];
                const double inv_nuT = 1.0 / r;
                const double ks = KScale<K>::v;
                const double* rt = out.rs + (int64_t)tg * DR;
                for (int j = 0; j < DU; ++j) {
                    double v = res[tt][j] + ks * accd[j];
                    for (int a = 0; a < DR; ++a) v -= out.self_val[j * DR + a] * inv_nuT * rt[a];
                    out.pot[(int64_t)oi * DU + j] = v;
                }
                if (GRAD && out.grad) {
                    const double in3 = inv_nuT * inv_nuT * inv_nuT;
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < DU; ++j) {
                            double v = res[tt][DU + i * DU + j] + ks * gaccd[i * DU + j];
                            for (int a = 0; a < DR; ++a) v -= out.self_grad[(i * DU + j) * DR + a] * in3 * rt[a];
                            out.grad[((int64_t)oi * 3 + i) * DU + j] = v;
                        }
                }
            }
        }
    }
}

}  // namespace dmk
