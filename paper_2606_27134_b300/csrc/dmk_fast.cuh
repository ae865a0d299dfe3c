// Kernels for p <= kMaxPFast that replace the generic versions in dmk_kernels.cuh:
//  * upward pass on 8-CTA thread-block clusters (one CTA per child octant, reduction of the
//    eight contributions through distributed shared memory) and the shift to children with one
//    CTA per (parent, child);
//  * translation + incoming plane-wave transform without materialising the weighted spectrum;
//  * the leaf stage, one thread per target, with in-support pair compaction.
//
// A p x p x p tensor sits in shared memory x-major with an odd row pitch P = p | 1, so that
// p-long fibers along any axis, one per thread, are read without bank conflicts.  Contracting
// one axis with a p x p operator is then "each thread owns one fiber": it reads its p inputs
// and accumulates p outputs in registers, with the operator rows loaded as shared-memory
// broadcasts.  Operator rows are zero-padded to MAXP so the unrolled loops need no guards.
#pragma once
#include <cooperative_groups.h>
#include <cuda_fp16.h>

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

// two fibers per thread: out0/out1[j] = sum_k M[k][j] in(fiber0/1, k); each operator row
// (read as four-vectors) serves both fibers
template <class T, int MAXP>
__device__ __forceinline__ void fiber_contract2(const T* in, int p, int P, int ax, int fa0, int fb0, int fa1,
                                                int fb1, bool two, const T* M, T (&acc0)[MAXP],
                                                T (&acc1)[MAXP]) {
    static_assert(MAXP % 4 == 0, "operator rows are read as four-vectors");
#pragma unroll
    for (int j = 0; j < MAXP; ++j) { acc0[j] = 0; acc1[j] = 0; }
    for (int k = 0; k < p; ++k) {
        const int e0 = (ax == 2) ? pidx(fa0, fb0, k, p, P) : (ax == 1) ? pidx(fa0, k, fb0, p, P) : pidx(k, fa0, fb0, p, P);
        const int e1 = (ax == 2) ? pidx(fa1, fb1, k, p, P) : (ax == 1) ? pidx(fa1, k, fb1, p, P) : pidx(k, fa1, fb1, p, P);
        const T x0 = in[e0];
        const T x1 = two ? in[e1] : T(0);
        const Quad<T>* row = reinterpret_cast<const Quad<T>*>(M + k * MAXP);
#pragma unroll
        for (int q = 0; q < MAXP / 4; ++q) {
            const Quad<T> m = row[q];
            acc0[4 * q] = fma(m.x, x0, acc0[4 * q]);
            acc0[4 * q + 1] = fma(m.y, x0, acc0[4 * q + 1]);
            acc0[4 * q + 2] = fma(m.z, x0, acc0[4 * q + 2]);
            acc0[4 * q + 3] = fma(m.w, x0, acc0[4 * q + 3]);
            acc1[4 * q] = fma(m.x, x1, acc1[4 * q]);
            acc1[4 * q + 1] = fma(m.y, x1, acc1[4 * q + 1]);
            acc1[4 * q + 2] = fma(m.z, x1, acc1[4 * q + 2]);
            acc1[4 * q + 3] = fma(m.w, x1, acc1[4 * q + 3]);
        }
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

// p^3 tensor from global memory into the padded shared layout: one p-long row per thread, all of
// its loads in flight at once (no index division)
template <class T, int MAXP = kMaxPFast>
__device__ __forceinline__ void load_padded_batched(T* dst, const T* __restrict__ src, int p, int P) {
    const int rows = p * p;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const T* s = src + (size_t)r * p;
        T v[MAXP];
#pragma unroll
        for (int j = 0; j < MAXP; ++j) v[j] = (j < p) ? s[j] : T(0);
#pragma unroll
        for (int j = 0; j < MAXP; ++j)
            if (j < p) dst[r * P + j] = v[j];
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


// Grid values -> Chebyshev coefficients in place, for leaves whose grid did not come through
// k_shift_child (root-level leaves, and every leaf when p > kMaxPFast).
template <class T>
__global__ void k_grid2coef(int ncap, const int* __restrict__ nleaf_dev, const int* __restrict__ boxes,
                            const int* __restrict__ level, int root_only, Tab<T> tab, T* __restrict__ local,
                            unsigned char* scratch, size_t per_cta, int use_smem) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, du = tab.d_u;
    const int n = min(ncap, *nleaf_dev);   // the first ncap entries of the leaf list at most
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
    __shared__ int sidx[kSrcChunk];
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
                        sidx[slot] = out.orig[si];
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
                        // r = 0 and the target's own periodic images (|p| >= nu_0) are dropped
                        if (r2 < snu2[k] && r2 > T(0) && sidx[k] != out.orig[t0 + tt]) q[cnt++][tt] = (unsigned char)k;
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
                        Pr::eval(ChebSeries<T>(tab, fits, r2, sinv[k]), dx, dy, dz, r2, sinv[k], sr[k], acc, gacc);
                    }
                    for (int j = 0; j < DU; ++j) accd[j] += (double)acc[j];
                    for (int j = 0; j < 3 * DU; ++j) gaccd[j] += (double)gacc[j];
                }
            }
            __syncthreads();
            // (4) self correction and write-back (FP64)
            if (act && out.perm[t0 + tt] < out.n_orig) {
                const int tg = t0 + tt;
                const int oi = out.perm[tg];
                const double inv_nuT = 1.0 / r;
                const double ks = KScale<K>::v;
                const double* rt = out.rs + (int64_t)tg * DR;
                for (int j = 0; j < DU; ++j) {
                    double v = res[tt][j] + ks * accd[j] + (out.ucst ? out.ucst[j] : 0.0);
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

namespace dmk {

// V(m) = sum over non-leaf colleagues C at offset d of exp(-i (2 pi/3) m.d) W_C(m), then
// component j of op(m) V (App. B symbols on the integer wave vector; see apply_op).  DR is the
// strength dimension, a template argument so that V stays in registers.
// Translation + difference-kernel symbol (Sec. 3.1.4), one thread per (non-leaf box, mode):
//   V(m) = 2^(a l) g(m) op(m) sum_C exp(-i (2 pi/3) m.d_C) W_C(m)
// over the non-leaf colleagues C (offset d_C).  The symbol -- the scalar 2^(a l) g(m) and the
// tensor op(m) of App. B mapping d_rho strength components to d_u -- depends on the mode only,
// so it commutes with the sum over colleagues.  For d_rho <= 3 it is applied after the sum
// (OP = true, NC = d_rho gathered components); for the stresslet (d_rho = 9, d_u = 3),
// k_pw_symbol applies it to every box's spectrum first, in place, so that the translation
// gathers 3 components instead of 9 (OP = false, NC = 3).  Each thread gathers its mode once
// for all output components.  Blocks are ordered (group of kTransGroup mode blocks, box, mode
// block) so that the boxes running together share their colleagues' spectra in L2.
constexpr int kTransThreads = 256;
constexpr int kTransGroup = 8;

// exp(-i (2 pi/3) r) for r = 0, 1, 2
template <class T>
__device__ __forceinline__ Cx<T> third_root(int r) {
    const T c3 = T(-0.5), s3 = T(-0.86602540378443864676);
    return (r == 0) ? Cx<T>{1, 0} : (r == 1 ? Cx<T>{c3, s3} : Cx<T>{c3, -s3});
}

template <class T, int NC, bool OP>
__global__ void __launch_bounds__(kTransThreads) k_pw_trans(int n, const int* __restrict__ nl_box, BoxArrays B,
                                                            Tab<T> tab, const Cx<T>* __restrict__ W, int wstride,
                                                            Cx<T>* __restrict__ Vw) {
    const int du = tab.d_u, nf = tab.nf, NF = tab.NF, nfh = tab.nfh;
    const int nW = NF * NF * nfh;
    const int nchunk = (nW + kTransThreads - 1) / kTransThreads;
    const int gsz = n * kTransGroup;
    const int grp = blockIdx.x / gsz, rem = blockIdx.x - grp * gsz;
    const int bi = rem / kTransGroup, chunk = grp * kTransGroup + rem % kTransGroup;
    if (chunk >= nchunk) return;
    __shared__ int ncol;
    __shared__ int col_nl[27];
    __shared__ int col_d[27];
    const int box = nl_box[bi];
    if (threadIdx.x < 32) {
        // the non-leaf colleagues in offset order, one lane per offset (ballot compaction)
        const int d = threadIdx.x;
        int C = -1;
        bool ok = false;
        if (d < 27) {
            C = B.coll[box * 27 + d];
            ok = C >= 0 && B.nl[C] >= 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const int k = __popc(bal & ((1u << d) - 1u));
            col_nl[k] = B.nl[C];
            col_d[k] = d;
        }
        if (d == 0) ncol = __popc(bal);
    }
    __syncthreads();
    const int e = chunk * kTransThreads + threadIdx.x;
    if (e >= nW) return;
    const int i1 = e / (NF * nfh), i2 = (e / nfh) % NF, m3 = e % nfh;
    const int m1 = i1 - nf, m2 = i2 - nf;
    // m mod 3 per axis, in 0..2
    const int r1 = ((m1 % 3) + 3) % 3, r2 = ((m2 % 3) + 3) % 3, r3 = m3 % 3;
    // colleagues in batches of KB, all loads of a batch issued before the first FMA
    constexpr int KB = NC == 1 ? 9 : 3;
    Cx<T> V[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) V[a] = {0, 0};
    const int nc = ncol;
    for (int k0 = 0; k0 < nc; k0 += KB) {
        Cx<T> w[KB][NC];
#pragma unroll
        for (int kk = 0; kk < KB; ++kk) {
            const int k = k0 + kk;
            const Cx<T>* Wc = W + (size_t)col_nl[k < nc ? k : 0] * wstride * nW + e;
#pragma unroll
            for (int a = 0; a < NC; ++a) w[kk][a] = (k < nc) ? Wc[(size_t)a * nW] : Cx<T>{0, 0};
        }
#pragma unroll
        for (int kk = 0; kk < KB; ++kk) {
            const int d = col_d[k0 + kk < nc ? k0 + kk : 0];
            const int t = r1 * (d % 3 - 1) + r2 * ((d / 3) % 3 - 1) + r3 * (d / 9 - 1) + 6;   // 0..12
            const Cx<T> ph = third_root<T>(t % 3);
#pragma unroll
            for (int a = 0; a < NC; ++a) cfma(V[a], ph, w[kk][a]);
        }
    }
    if constexpr (OP) {
        const T gs = pow2t<T>(tab.level_power * B.level[box]) * tab.gdiff[e];
        Cx<T> out[3];
        if constexpr (NC == 1) {
            out[0] = V[0];
        } else {
            const T mv[3] = {(T)m1, (T)m2, (T)m3};
            apply_op<T>(tab.kernel, mv, V, out);
        }
        for (int j = 0; j < du; ++j) Vw[((size_t)bi * du + j) * nW + e] = {gs * out[j].x, gs * out[j].y};
    } else {
#pragma unroll
        for (int j = 0; j < NC; ++j) Vw[((size_t)bi * NC + j) * nW + e] = V[j];
    }
}

// The symbol 2^(a l) g(m) op(m) applied to every non-leaf box's outgoing spectrum in place: the
// d_u results overwrite the first d_u of the d_rho component slots (thread per (box, mode); each
// thread reads its own d_rho values before it writes).  Used for the stresslet (d_rho = 9).
template <class T, int DR>
__global__ void __launch_bounds__(kTransThreads) k_pw_symbol(int n, const int* __restrict__ nl_box, BoxArrays B,
                                                             Tab<T> tab, Cx<T>* __restrict__ W) {
    const int nf = tab.nf, NF = tab.NF, nfh = tab.nfh, du = tab.d_u;
    const int nW = NF * NF * nfh;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nW) return;
    const int bi = (int)(t / nW), e = (int)(t - (int64_t)bi * nW);
    const int i1 = e / (NF * nfh), i2 = (e / nfh) % NF, m3 = e % nfh;
    const T mv[3] = {(T)(i1 - nf), (T)(i2 - nf), (T)m3};
    Cx<T>* Wb = W + (size_t)bi * DR * nW + e;
    Cx<T> V[DR];
#pragma unroll
    for (int a = 0; a < DR; ++a) V[a] = Wb[(size_t)a * nW];
    Cx<T> out[3];
    apply_op<T>(tab.kernel, mv, V, out);
    const T gs = pow2t<T>(tab.level_power * B.level[nl_box[bi]]) * tab.gdiff[e];
    for (int j = 0; j < du; ++j) Wb[(size_t)j * nW] = {gs * out[j].x, gs * out[j].y};
}

// Plane-wave outgoing expansions with the symmetries of the nodes and of the modes (Sec.
// 3.1.4, Eq. Dl_int_discr): W(m) = sum_j proxy(j) exp(-i theta m . eta_j), theta = pi / 3,
// m3 >= 0 only (real input).  With C(m, k) = cos(theta m eta_k) and S(m, k) = sin(theta m eta_k),
// the first-kind nodes satisfy eta_{p-1-k} = -eta_k, so along one axis C is even and S odd
// about the middle node, and in m C is even and S odd.  One 1-D stage on a complex column
// A = R - i I (I = 0 for the first, real, stage) then reads, with the even and odd parts
// Re_k = R_k + R_{p-1-k}, Ro_k = R_k - R_{p-1-k} (Ie, Io likewise; k < p/2, plus the middle
// node eta = 0 for odd p):
//   P = sum Re C, Q = sum Io S, U = sum Ro S, V = sum Ie C,
//   A'(+m) = (P - Q) - i (U + V),   A'(-m) = (P + Q) - i (V - U),
// i.e. p real FMA per complex output instead of 4 p.  Stage 1 (j3 -> m3 >= 0, thread per (j1,
// j2) fiber), stage 2 (j2 -> m2, thread per (j1, m3) column, the range of |m2| split in nsplit
// parts when shared memory is short), stage 3 (j1 -> m1, thread per (m2, m3) column), real
// parts in separate arrays.  Work item = (box, part of |m2|); stage 1 is repeated per part.
template <class T>
constexpr int pw_sym_threads() { return sizeof(T) == 4 ? 512 : 256; }

template <class T, int MH>
__global__ void __launch_bounds__(pw_sym_threads<T>(), 1) k_pwout3(int n, const int* __restrict__ nl_box, Tab<T> tab,
                                                   const T* __restrict__ proxy, Cx<T>* __restrict__ W, int nsplit) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, P = odd_pitch(p), drho = tab.d_rho;
    const int nf = tab.nf, NF = tab.NF, nfh = tab.nfh, nW = NF * NF * nfh;
    const int hp = p >> 1, odd = p & 1, pm3 = nfh | 1;
    const int hcn = (nfh + nsplit - 1) / nsplit;            // |m2| values per part
    T* Ct = reinterpret_cast<T*>(dsmem);                     // hp x MH: C(m, k) at [k][m]
    T* St = Ct + hp * MH;                                    // hp x MH: S(m, k)
    T* R1 = St + hp * MH;                                    // p^2 x pm3
    T* I1 = R1 + p2 * pm3;
    T* R2 = I1 + p2 * pm3;                                   // p x (2 hcn) x nfh, slot = 2 i + (m2 < 0)
    T* I2 = R2 + p * 2 * hcn * nfh;
    T* X = R2;                                               // p^2 x P (stage 1 input), aliases R2/I2
    for (int e = threadIdx.x; e < hp * MH; e += blockDim.x) {
        const int k = e / MH, m = e % MH;
        const Cx<T> v = (m < nfh) ? tab.E[(m + nf) * p + k] : Cx<T>{0, 0};   // exp(-i theta m eta_k)
        Ct[e] = v.x;
        St[e] = -v.y;
    }
    for (int w = blockIdx.x; w < nsplit * n; w += gridDim.x) {
        const int bi = w / nsplit, part = w % nsplit;
        const int a0 = part * hcn, hc = min(hcn, nfh - a0);
        if (hc <= 0) continue;
        const int box = nl_box[bi];
        for (int a = 0; a < drho; ++a) {
            __syncthreads();
            load_padded_batched<T, kMaxPFast>(X, proxy + ((size_t)box * drho + a) * p3, p, P);
            __syncthreads();
            // stage 1: j3 -> m3, real input
            for (int c = threadIdx.x; c < p2; c += blockDim.x) {
                T ev[kMaxPFast / 2], od[kMaxPFast / 2];
#pragma unroll
                for (int k = 0; k < kMaxPFast / 2; ++k) {
                    const T x0 = (k < hp) ? X[c * P + k] : T(0), x1 = (k < hp) ? X[c * P + p - 1 - k] : T(0);
                    ev[k] = x0 + x1;
                    od[k] = x0 - x1;
                }
                const T mid = odd ? X[c * P + hp] : T(0);
                T r[MH], im[MH];
#pragma unroll
                for (int m = 0; m < MH; ++m) { r[m] = mid; im[m] = 0; }
#pragma unroll
                for (int k = 0; k < kMaxPFast / 2; ++k) {
                    if (k < hp) {
                        const Quad<T>* cr = reinterpret_cast<const Quad<T>*>(Ct + k * MH);
                        const Quad<T>* sr = reinterpret_cast<const Quad<T>*>(St + k * MH);
#pragma unroll
                        for (int q = 0; q < MH / 4; ++q) {
                            const Quad<T> cv = cr[q], sv = sr[q];
                            r[4 * q] = fma(ev[k], cv.x, r[4 * q]);
                            r[4 * q + 1] = fma(ev[k], cv.y, r[4 * q + 1]);
                            r[4 * q + 2] = fma(ev[k], cv.z, r[4 * q + 2]);
                            r[4 * q + 3] = fma(ev[k], cv.w, r[4 * q + 3]);
                            im[4 * q] = fma(od[k], sv.x, im[4 * q]);
                            im[4 * q + 1] = fma(od[k], sv.y, im[4 * q + 1]);
                            im[4 * q + 2] = fma(od[k], sv.z, im[4 * q + 2]);
                            im[4 * q + 3] = fma(od[k], sv.w, im[4 * q + 3]);
                        }
                    }
                }
#pragma unroll
                for (int m = 0; m < MH; ++m)
                    if (m < nfh) { R1[c * pm3 + m] = r[m]; I1[c * pm3 + m] = im[m]; }
            }
            __syncthreads();
            // stage 2: j2 -> m2 for |m2| in [a0, a0 + hc), both signs
            for (int c = threadIdx.x; c < p * nfh; c += blockDim.x) {
                const int j1 = c / nfh, m3 = c % nfh;
                const T* r1 = R1 + (size_t)j1 * p * pm3 + m3;
                const T* i1 = I1 + (size_t)j1 * p * pm3 + m3;
                T Pa[MH], Qa[MH], Ua[MH], Va[MH];
                const T rm = odd ? r1[hp * pm3] : T(0), im_ = odd ? i1[hp * pm3] : T(0);
#pragma unroll
                for (int m = 0; m < MH; ++m) { Pa[m] = rm; Va[m] = im_; Qa[m] = 0; Ua[m] = 0; }
                for (int k = 0; k < hp; ++k) {
                    const T ra = r1[k * pm3], rb = r1[(p - 1 - k) * pm3];
                    const T ia = i1[k * pm3], ib = i1[(p - 1 - k) * pm3];
                    const T re = ra + rb, ro = ra - rb, ie = ia + ib, io = ia - ib;
                    const T* cr = Ct + k * MH + a0;
                    const T* sr = St + k * MH + a0;
#pragma unroll
                    for (int m = 0; m < MH; ++m) {
                        if (m < hc) {
                            const T cv = cr[m], sv = sr[m];
                            Pa[m] = fma(re, cv, Pa[m]);
                            Va[m] = fma(ie, cv, Va[m]);
                            Qa[m] = fma(io, sv, Qa[m]);
                            Ua[m] = fma(ro, sv, Ua[m]);
                        }
                    }
                }
#pragma unroll
                for (int m = 0; m < MH; ++m) {
                    if (m < hc) {
                        const int sp = ((j1 * 2 * hcn) + 2 * m) * nfh + m3, sm = sp + nfh;
                        R2[sp] = Pa[m] - Qa[m];
                        I2[sp] = Ua[m] + Va[m];
                        R2[sm] = Pa[m] + Qa[m];
                        I2[sm] = Va[m] - Ua[m];
                    }
                }
            }
            __syncthreads();
            // stage 3: j1 -> m1, all m1, written to W[nl][a][(m1 NF + m2) nfh + m3]
            Cx<T>* out = W + ((size_t)bi * drho + a) * nW;
            for (int c = threadIdx.x; c < 2 * hc * nfh; c += blockDim.x) {
                const int slot = c / nfh, m3 = c % nfh;
                const int mi = slot >> 1, neg = slot & 1;
                const int m2 = neg ? -(a0 + mi) : (a0 + mi);
                if (neg && m2 == 0) continue;
                const T* r2 = R2 + (size_t)slot * nfh + m3;
                const T* i2 = I2 + (size_t)slot * nfh + m3;
                const int cs = 2 * hcn * nfh;                    // stride of j1
                T Pa[MH], Qa[MH], Ua[MH], Va[MH];
                const T rm = odd ? r2[hp * cs] : T(0), im_ = odd ? i2[hp * cs] : T(0);
#pragma unroll
                for (int m = 0; m < MH; ++m) { Pa[m] = rm; Va[m] = im_; Qa[m] = 0; Ua[m] = 0; }
                for (int k = 0; k < hp; ++k) {
                    const T ra = r2[k * cs], rb = r2[(p - 1 - k) * cs];
                    const T ia = i2[k * cs], ib = i2[(p - 1 - k) * cs];
                    const T re = ra + rb, ro = ra - rb, ie = ia + ib, io = ia - ib;
                    const Quad<T>* cr = reinterpret_cast<const Quad<T>*>(Ct + k * MH);
                    const Quad<T>* sr = reinterpret_cast<const Quad<T>*>(St + k * MH);
#pragma unroll
                    for (int q = 0; q < MH / 4; ++q) {
                        const Quad<T> cv = cr[q], sv = sr[q];
                        const T cc[4] = {cv.x, cv.y, cv.z, cv.w}, ss[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            Pa[4 * q + u] = fma(re, cc[u], Pa[4 * q + u]);
                            Va[4 * q + u] = fma(ie, cc[u], Va[4 * q + u]);
                            Qa[4 * q + u] = fma(io, ss[u], Qa[4 * q + u]);
                            Ua[4 * q + u] = fma(ro, ss[u], Ua[4 * q + u]);
                        }
                    }
                }
                const size_t col = (size_t)(m2 + nf) * nfh + m3;
#pragma unroll
                for (int m = 0; m < MH; ++m) {
                    if (m < nfh) {
                        // W = R - i I with R, I the real and (minus) imaginary parts
                        out[(size_t)(m + nf) * NF * nfh + col] = {Pa[m] - Qa[m], -(Ua[m] + Va[m])};
                        if (m > 0) out[(size_t)(nf - m) * NF * nfh + col] = {Pa[m] + Qa[m], -(Va[m] - Ua[m])};
                    }
                }
            }
        }
    }
}

// shared memory of k_pwout3 for nsplit parts of |m2|
template <class T>
inline size_t pwout3_smem(int p, int nfh, int MH, int nsplit) {
    const int hp = p / 2, pm3 = nfh | 1, P = p | 1, hcn = (nfh + nsplit - 1) / nsplit;
    const size_t r2 = (size_t)2 * p * 2 * hcn * nfh, x = (size_t)p * p * P;
    return ((size_t)2 * hp * MH + (size_t)2 * p * p * pm3 + std::max(r2, x)) * sizeof(T);
}

// Incoming transform with the same symmetries (Sec. 3.1.4): u(j) += Re sum_m w(m3) V(m)
// exp(+i theta m . eta_j) over the half spectrum m3 >= 0 (w = 1 for m3 = 0, else 2).  Along
// one axis, for a complex column V(m) = a_m + i b_m, V(-m) = c_m + i d_m and the mirrored node
// pair (k, p-1-k):
//   Ap = sum (a+c) C, Bp = sum (b+d) C, As = sum (a-c) S, Bs = sum (b-d) S   (m >= 0; V(0) once)
//   B(k) = (Ap - Bs) + i (Bp + As),   B(p-1-k) = (Ap + Bs) + i (Bp - As),
// the middle node (odd p) taking sum (a+c) + i sum (b+d).  Stage A (m1 -> j1, thread per (m2,
// m3) column read from global memory), stage B (m2 -> j2, thread per (j1, m3)), stage C (m3 ->
// j3, real part with the weights, thread per (j1, j2) fiber), real parts in separate arrays.
template <class T, int MH>
__global__ void __launch_bounds__(pw_sym_threads<T>(), 1) k_pwin4(int n, const int* __restrict__ nl_box, Tab<T> tab,
                                                  const Cx<T>* __restrict__ Vw, T* __restrict__ local) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, du = tab.d_u;
    const int nf = tab.nf, NF = tab.NF, nfh = tab.nfh, nW = NF * NF * nfh;
    const int hp = p >> 1, odd = p & 1, pm3 = nfh | 1;
    constexpr int HPM = kMaxPFast / 2;
    T* Ct = reinterpret_cast<T*>(dsmem);                     // MH x HPM: C(m, k) at [m][k]
    T* St = Ct + MH * HPM;
    T* Ar = St + MH * HPM;                                   // p x NF x nfh: stage A output
    T* Ai = Ar + (size_t)p * NF * nfh;
    T* Br = Ai + (size_t)p * NF * nfh;                       // p^2 x pm3: stage B output
    T* Bi = Br + (size_t)p2 * pm3;
    for (int e = threadIdx.x; e < MH * HPM; e += blockDim.x) {
        const int m = e / HPM, k = e % HPM;
        const Cx<T> v = (m < nfh && k < hp) ? tab.E[(m + nf) * p + k] : Cx<T>{0, 0};
        Ct[e] = v.x;
        St[e] = -v.y;
    }
    for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const int box = nl_box[bi];
        for (int j = 0; j < du; ++j) {
            __syncthreads();
            const Cx<T>* V = Vw + ((size_t)bi * du + j) * nW;
            // stage A: m1 -> j1 for every (m2, m3) column
            for (int c = threadIdx.x; c < NF * nfh; c += blockDim.x) {
                T Ap[HPM + 1], Bp[HPM + 1], As[HPM], Bs[HPM];
#pragma unroll
                for (int k = 0; k <= HPM; ++k) { Ap[k] = 0; Bp[k] = 0; }
#pragma unroll
                for (int k = 0; k < HPM; ++k) { As[k] = 0; Bs[k] = 0; }
                for (int m = 0; m < nfh; ++m) {
                    const Cx<T> vp = V[(size_t)(nf + m) * NF * nfh + c];
                    const Cx<T> vm = (m > 0) ? V[(size_t)(nf - m) * NF * nfh + c] : Cx<T>{0, 0};
                    const T sa = vp.x + vm.x, sb = vp.y + vm.y, da = vp.x - vm.x, db = vp.y - vm.y;
                    const T* cr = Ct + m * HPM;
                    const T* sr = St + m * HPM;
#pragma unroll
                    for (int k = 0; k < HPM; ++k) {
                        const T cv = cr[k], sv = sr[k];
                        Ap[k] = fma(sa, cv, Ap[k]);
                        Bp[k] = fma(sb, cv, Bp[k]);
                        As[k] = fma(da, sv, As[k]);
                        Bs[k] = fma(db, sv, Bs[k]);
                    }
                    Ap[HPM] += sa;                             // middle node (odd p)
                    Bp[HPM] += sb;
                }
                const int i2 = c / nfh, m3 = c % nfh;
#pragma unroll
                for (int k = 0; k < HPM; ++k) {
                    if (k < hp) {
                        const size_t o0 = ((size_t)k * NF + i2) * nfh + m3, o1 = ((size_t)(p - 1 - k) * NF + i2) * nfh + m3;
                        Ar[o0] = Ap[k] - Bs[k];
                        Ai[o0] = Bp[k] + As[k];
                        Ar[o1] = Ap[k] + Bs[k];
                        Ai[o1] = Bp[k] - As[k];
                    }
                }
                if (odd) {
                    const size_t om = ((size_t)hp * NF + i2) * nfh + m3;
                    Ar[om] = Ap[HPM];
                    Ai[om] = Bp[HPM];
                }
            }
            __syncthreads();
            // stage B: m2 -> j2 for every (j1, m3)
            for (int c = threadIdx.x; c < p * nfh; c += blockDim.x) {
                const int j1 = c / nfh, m3 = c % nfh;
                const T* ar = Ar + (size_t)j1 * NF * nfh + m3;
                const T* ai = Ai + (size_t)j1 * NF * nfh + m3;
                T Ap[HPM + 1], Bp[HPM + 1], As[HPM], Bs[HPM];
#pragma unroll
                for (int k = 0; k <= HPM; ++k) { Ap[k] = 0; Bp[k] = 0; }
#pragma unroll
                for (int k = 0; k < HPM; ++k) { As[k] = 0; Bs[k] = 0; }
                for (int m = 0; m < nfh; ++m) {
                    const T pa = ar[(nf + m) * nfh], pb = ai[(nf + m) * nfh];
                    const T ma = (m > 0) ? ar[(nf - m) * nfh] : T(0), mb = (m > 0) ? ai[(nf - m) * nfh] : T(0);
                    const T sa = pa + ma, sb = pb + mb, da = pa - ma, db = pb - mb;
                    const T* cr = Ct + m * HPM;
                    const T* sr = St + m * HPM;
#pragma unroll
                    for (int k = 0; k < HPM; ++k) {
                        const T cv = cr[k], sv = sr[k];
                        Ap[k] = fma(sa, cv, Ap[k]);
                        Bp[k] = fma(sb, cv, Bp[k]);
                        As[k] = fma(da, sv, As[k]);
                        Bs[k] = fma(db, sv, Bs[k]);
                    }
                    Ap[HPM] += sa;
                    Bp[HPM] += sb;
                }
#pragma unroll
                for (int k = 0; k < HPM; ++k) {
                    if (k < hp) {
                        const size_t o0 = ((size_t)j1 * p + k) * pm3 + m3, o1 = ((size_t)j1 * p + p - 1 - k) * pm3 + m3;
                        Br[o0] = Ap[k] - Bs[k];
                        Bi[o0] = Bp[k] + As[k];
                        Br[o1] = Ap[k] + Bs[k];
                        Bi[o1] = Bp[k] - As[k];
                    }
                }
                if (odd) {
                    const size_t om = ((size_t)j1 * p + hp) * pm3 + m3;
                    Br[om] = Ap[HPM];
                    Bi[om] = Bp[HPM];
                }
            }
            __syncthreads();
            // stage C: m3 -> j3, real part with the half-spectrum weights
            T* u = local + ((size_t)box * du + j) * p3;
            for (int c = threadIdx.x; c < p2; c += blockDim.x) {
                const T* br = Br + (size_t)c * pm3;
                const T* bim = Bi + (size_t)c * pm3;
                T X1[HPM + 1], X2[HPM];
#pragma unroll
                for (int k = 0; k <= HPM; ++k) X1[k] = 0;
#pragma unroll
                for (int k = 0; k < HPM; ++k) X2[k] = 0;
                for (int m = 0; m < nfh; ++m) {
                    const T wgt = (m == 0) ? T(1) : T(2);
                    const T a = wgt * br[m], b = wgt * bim[m];
                    const T* cr = Ct + m * HPM;
                    const T* sr = St + m * HPM;
#pragma unroll
                    for (int k = 0; k < HPM; ++k) {
                        X1[k] = fma(a, cr[k], X1[k]);
                        X2[k] = fma(b, sr[k], X2[k]);
                    }
                    X1[HPM] += a;
                }
                T* uc = u + (size_t)c * p;
#pragma unroll
                for (int k = 0; k < HPM; ++k) {
                    if (k < hp) {
                        uc[k] += X1[k] - X2[k];
                        uc[p - 1 - k] += X1[k] + X2[k];
                    }
                }
                if (odd) uc[hp] += X1[HPM];
            }
        }
    }
}

template <class T>
inline size_t pwin4_smem(int p, int NF, int nfh, int MH) {
    const int pm3 = nfh | 1;
    return ((size_t)2 * MH * (kMaxPFast / 2) + (size_t)2 * p * NF * nfh + (size_t)2 * p * p * pm3) * sizeof(T);
}

}  // namespace dmk

namespace dmk {

// ------------------------------------------------------------------------------------------
// Helpers of the leaf stage for p <= kMaxPFast (k_pair, k_leafexp below).
// (a_h + a_l) + (b_h + b_l) as an unnormalised FP32 pair: the leading sum with its exact
// rounding error (Knuth's TwoSum), plus the trailing parts.  Accurate to about 2^-48 of the
// operands' magnitude.
__device__ __forceinline__ void two_float_add(float ah, float al, float bh, float bl, float& h, float& l) {
    const float s = ah + bh;
    const float bb = s - ah;
    const float e = (ah - (s - bb)) + (bh - bb);
    h = s;
    l = e + (al + bl);
}

// FP64 value as leading + trailing FP32 parts
__device__ __forceinline__ void split_double(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// Tensor-product Chebyshev sum at one target (Sec. 3.1.5): S = sum c[n1][n2][n3] T_n1(x) T_n2(y)
// T_n3(z) and its three derivatives, with c staged in shared memory in rows of NG four-vectors
// (n3 padded to 4 NG with zeros) and T_n3(z), T'_n3(z) in registers; the x and y recurrences run
// on the fly.  GUARD: rows shorter than NG four-vectors (ng < NG).
template <class T, int NG, bool GUARD, bool GRAD>
__device__ __forceinline__ void cheb_eval(const T* cs, int p, int ng, const T (&Tz)[kMaxPFast],
                                          const T (&dTz)[kMaxPFast], const T xi[3], T& S, T& Sx, T& Sy, T& Sz) {
    using Q4 = Quad<T>;
    T xm2 = 0, xm1 = 1, xu2 = 0, xu1 = 1;
    for (int n1 = 0; n1 < p; ++n1) {
        T tx, dtx;
        if (n1 == 0) { tx = 1; dtx = 0; }
        else if (n1 == 1) { tx = xi[0]; dtx = 1; xm2 = 1; xm1 = xi[0]; xu2 = 1; xu1 = 2 * xi[0]; }
        else {
            tx = 2 * xi[0] * xm1 - xm2;
            dtx = (T)n1 * xu1;
            const T un = 2 * xi[0] * xu1 - xu2;
            xm2 = xm1; xm1 = tx; xu2 = xu1; xu1 = un;
        }
        T b0 = 0, b1 = 0, b2 = 0;
        T ym2 = 0, ym1 = 1, yu2 = 0, yu1 = 1;
        const Q4* rows = reinterpret_cast<const Q4*>(cs + (size_t)n1 * p * 4 * ng);
        for (int n2 = 0; n2 < p; ++n2) {
            T ty, dty;
            if (n2 == 0) { ty = 1; dty = 0; }
            else if (n2 == 1) { ty = xi[1]; dty = 1; ym2 = 1; ym1 = xi[1]; yu2 = 1; yu1 = 2 * xi[1]; }
            else {
                ty = 2 * xi[1] * ym1 - ym2;
                dty = (T)n2 * yu1;
                const T un = 2 * xi[1] * yu1 - yu2;
                ym2 = ym1; ym1 = ty; yu2 = yu1; yu1 = un;
            }
            const Q4* row = rows + n2 * ng;
            T a0 = 0, a1 = 0, a0b = 0, a1b = 0;
#pragma unroll
            for (int gq = 0; gq < NG; ++gq) {
                if (!GUARD || gq < ng) {
                    const Q4 cv = row[gq];
                    a0 = fma(cv.x, Tz[4 * gq], a0);
                    a0b = fma(cv.y, Tz[4 * gq + 1], a0b);
                    a0 = fma(cv.z, Tz[4 * gq + 2], a0);
                    a0b = fma(cv.w, Tz[4 * gq + 3], a0b);
                    if (GRAD) {
                        a1 = fma(cv.x, dTz[4 * gq], a1);
                        a1b = fma(cv.y, dTz[4 * gq + 1], a1b);
                        a1 = fma(cv.z, dTz[4 * gq + 2], a1);
                        a1b = fma(cv.w, dTz[4 * gq + 3], a1b);
                    }
                }
            }
            a0 += a0b;
            b0 = fma(ty, a0, b0);
            if (GRAD) {
                a1 += a1b;
                b1 = fma(dty, a0, b1);
                b2 = fma(ty, a1, b2);
            }
        }
        S = fma(tx, b0, S);
        if (GRAD) {
            Sx = fma(dtx, b0, Sx);
            Sy = fma(tx, b1, Sy);
            Sz = fma(tx, b2, Sz);
        }
    }
}

// ------------------------------------------------------------------------------------------
// Leaf stage for p <= kMaxPFast in two launches.
//
// k_pair: the residual sums (Sec. 2.4 and the direct interactions of Sec. 3.1.5) as
// independent warp tasks.  A task is a tile of m consecutive targets of one leaf (m = kPairTile
// for the full tiles, and for the remainder one tile per set bit, so that every lane has a
// target); lane = s m + i holds target i and takes every S-th source (S = 32/m, split s); the S
// partial sums are combined by a fixed xor-shuffle tree.  Warps take tasks from a device
// counter, so no barrier couples the warps of a block.
//   Sources stream through the direct-list entries in order, 32 at a time (one per lane).  A
// lane forms its source's offset from the target leaf's centre (FP32 leading and trailing
// parts in the FP32 path) and tests it against the tile's bounding box expanded by the entry's
// nu: only a source within nu of the box can be within nu of a target of the tile.  The
// survivors (about 40% of the sources of a 16-target tile, against 15% inside the support of
// one target for uniform points) are appended in order to the warp's ring of kPairList records
// ((x, y, z, nu^2), (x_lo, y_lo, z_lo, 1/nu), strengths); each full block of 32 survivors is
// then evaluated by every lane for its own target -- broadcast shared-memory reads, no per-lane
// queue -- with two-float differences, the exact test 0 < r^2 < nu^2 (r = 0 is the target
// itself, Eq. periodic_sum drops it; the target's own periodic images lie at |p| >= nu_0 and
// are dropped by the index of the original point) and the cubic residual tables.  Images of a
// non-exact tiling are sources; their own sums are not written.  FP32 partial sums are
// folded into a two-float accumulator per block (FP64 in the FP64 path); the order of every
// sum is fixed, so results are reproducible.  The result K * sum is written in input order.
// The kernel needs only the tree, so it may run beside the far field on another stream.
//
// k_leafexp: thread per target.  The leaf's Chebyshev coefficients c[n1][n2][n3] (x, y, z) are
// staged in shared memory with the n3 rows padded to a multiple of four; each thread keeps
// T_n3(z), T'_n3(z) in registers, runs the y and x recurrences on the fly and reads coefficient
// rows as broadcast vectors (Sec. 3.1.5).  The expansion is added to the residual sums written
// by k_pair, the self term (Sec. 2.4) subtracted, and the result written in FP64.
constexpr int kPairWarps = 4;
constexpr int kPairList = 64;      // survivor ring per warp (two blocks of 32)

// byte offsets within one warp's shared-memory region of k_pair
template <class T, int DR>
struct PairSmem {
    static constexpr size_t a = 0;                                                    // Quad<T> [kPairList]
    static constexpr size_t b = a + kPairList * sizeof(Quad<T>);                      // Quad<T> [kPairList]
    static constexpr size_t r = b + kPairList * sizeof(Quad<T>);                      // T [kPairList][DR]
    static constexpr size_t i = r + kPairList * DR * sizeof(T);                       // int [kPairList]
    static constexpr size_t bytes = (i + kPairList * sizeof(int) + 15) & ~(size_t)15;
};

// hi + lo += v (Knuth's TwoSum on the leading part)
__device__ __forceinline__ void two_float_acc(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}

template <class T, int K, bool GRAD>
__global__ void __launch_bounds__(kPairWarps * 32, sizeof(T) == 4 ? (K == DMK_LAPLACE ? 6 : 4) : 2) k_pair(const int* __restrict__ leaves, BoxArrays B, Tab<T> tab,
                                                            Geo g, const double* __restrict__ xs, int64_t N,
                                                            const int* __restrict__ doffs,
                                                            const int* __restrict__ toffs, int tcap,
                                                            const int4* __restrict__ tasks, int* __restrict__ next,
                                                            const DirectEntry* __restrict__ dl, LeafOut out) {
    using Pr = Pair<T, K, GRAD>;
    using Q4 = Quad<T>;
    constexpr int DR = Pr::DR, DU = Pr::DU, NA = DU + (GRAD ? 3 * DU : 0);
    constexpr bool kTwo = sizeof(T) == 4;
    constexpr int RQ = point_record_floats(DR) / 4;     // float4s per point record
    using WS = PairSmem<T, DR>;
    constexpr int NSER = (K == DMK_STRESSLET) ? (GRAD ? 6 : 3) : ((GRAD && K != DMK_LAPLACE) ? 5 : 2);
    __shared__ Quad<float> herm[kTwo ? NSER * kHermNT : 1];
    __shared__ T fits[kTwo ? 1 : 256];
    extern __shared__ __align__(16) unsigned char dsmp[];
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu, below = (1u << lane) - 1u;
    unsigned char* wsm = dsmp + (threadIdx.x >> 5) * WS::bytes;
    Q4* sA = reinterpret_cast<Q4*>(wsm + WS::a);
    Q4* sB = reinterpret_cast<Q4*>(wsm + WS::b);
    T (*sr)[DR] = reinterpret_cast<T (*)[DR]>(wsm + WS::r);
    int* sI = reinterpret_cast<int*>(wsm + WS::i);
    if constexpr (kTwo) {
        const Quad<float>* hsrc = reinterpret_cast<const Quad<float>*>(tab.herm);
        for (int e = threadIdx.x; e < NSER * kHermNT; e += blockDim.x) herm[e] = hsrc[e];
    } else {
        for (int e = threadIdx.x; e < min(256, tab.n_q + tab.n_f + tab.n_g + tab.n_dq + tab.n_df + tab.n_dg);
             e += blockDim.x)
            fits[e] = tab.fit[e];
    }
    __syncthreads();
    const int ntask = toffs[tcap] - toffs[0];
    const double inv_s = 1.0 / g.s, s2 = g.s * g.s;
    const float inv_s_f = (float)inv_s, s2_f = (float)s2;
    // the box test passes every source within nu of the tile's box: its FP32 rounding (relative
    // 1e-6 at most for offsets below 3 nu) is covered by the factor on nu^2
    const T box_margin = kTwo ? T(1.0001) : T(1.0 + 1e-12);
    float Lh[3], Ll[3], s_hi, s_lo;
    for (int a = 0; a < 3; ++a) split_double(g.L[a], Lh[a], Ll[a]);
    split_double(g.s, s_hi, s_lo);
    while (true) {
        int t = 0;
        if (lane == 0) t = atomicAdd(next, 1);
        t = __shfl_sync(full, t, 0);
        if (t >= ntask) break;
        const int4 tk = tasks[t];
        const int li = tk.x, m = tk.z;
        const int lgm = __ffs(m) - 1;
        const int ti = lane & (m - 1), s = lane >> lgm, S = 32 >> lgm;
        const int box = leaves[li];
        const int l = B.level[box];
        // minus the leaf centre c = (2 ix + 1) s 2^(-l-1), as leading + trailing FP32 parts
        // (two-product of the odd integer with s's parts: exact to 2^-48 of c, no FP64)
        float ch[3], cl[3];
        double c[3];
        if constexpr (kTwo) {
            const float sc = pow2f(-l - 1);
            for (int a = 0; a < 3; ++a) {
                const float k = (float)(2 * B.ix[3 * box + a] + 1);
                const float hi = k * s_hi;
                const float lo = fmaf(k, s_hi, -hi) + k * s_lo;
                two_float_add(-hi * sc, -lo * sc, 0.f, 0.f, ch[a], cl[a]);
            }
        } else {
            const double r = ldexp(g.s, -l);
            for (int a = 0; a < 3; ++a) c[a] = (B.ix[3 * box + a] + 0.5) * r;
        }
        const int tg = B.start[box] + tk.y + ti;
        const int tgo = out.orig[tg];                  // the original point the target is
        T xt[3], xtl[3] = {0, 0, 0};
        if constexpr (kTwo) {
            const float4 p0 = out.pk[(int64_t)tg * RQ], p1 = out.pk[(int64_t)tg * RQ + 1];
            two_float_add(p0.x, p1.x, ch[0], cl[0], xt[0], xtl[0]);
            two_float_add(p0.y, p1.y, ch[1], cl[1], xt[1], xtl[1]);
            two_float_add(p0.z, p1.z, ch[2], cl[2], xt[2], xtl[2]);
        } else {
            for (int a = 0; a < 3; ++a) xt[a] = (T)(xs[a * N + tg] - c[a]);
        }
        // the tile's bounding box (lanes of one split hold the m targets)
        T blo[3], bhi[3];
        for (int a = 0; a < 3; ++a) blo[a] = bhi[a] = xt[a] + xtl[a];
        for (int o = 1; o < m; o <<= 1)
            for (int a = 0; a < 3; ++a) {
                blo[a] = min(blo[a], __shfl_xor_sync(full, blo[a], o));
                bhi[a] = max(bhi[a], __shfl_xor_sync(full, bhi[a], o));
            }
        // two-float (FP32 path) or FP64 accumulators, FP32 partial sums per block of survivors
        T acc_hi[NA], acc_lo[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) { acc_hi[j] = 0; acc_lo[j] = 0; }
        int head = 0, tail = 0;
        // the target's own periodic images can pass the rounded support test only in an entry of
        // level 0 with an image shift (|p| >= nu_0 = nu there); elsewhere |p| >= 2 nu and the test
        // alone drops them, so the index comparison runs only once such an entry was seen
        bool chk = false;
        // evaluates the survivors head .. head + cnt - 1 of the ring for this lane's target
        auto run_block = [&](int cnt) {
            __syncwarp();
            T acc[DU], gacc[3 * DU];
#pragma unroll
            for (int j = 0; j < DU; ++j) acc[j] = 0;
#pragma unroll
            for (int j = 0; j < 3 * DU; ++j) gacc[j] = 0;
            if constexpr (kTwo) {
                // FP32: every lane evaluates the block's survivors in order (broadcast reads),
                // predicated on its own support test
#pragma unroll 2
                for (int i = s; i < cnt; i += S) {
                    const int k = (head + i) & (kPairList - 1);
                    const Q4 a = sA[k], b = sB[k];
                    T dx = xt[0] - a.x, dy = xt[1] - a.y, dz = xt[2] - a.z;
                    dx += xtl[0] - b.x;
                    dy += xtl[1] - b.y;
                    dz += xtl[2] - b.z;
                    const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    // r = 0 (the target itself at p = 0, or a coincident point) and the target's
                    // own periodic images (|p| >= nu_0 >= nu: outside the support, however r^2
                    // rounds) are dropped
                    if (chk) {
                        if (r2 > T(0) && r2 < a.w && sI[k] != tgo)
                            Pr::eval(HermSeries(herm, r2, b.w), dx, dy, dz, r2, b.w, sr[k], acc, gacc);
                    } else {
                        if (r2 > T(0) && r2 < a.w)
                            Pr::eval(HermSeries(herm, r2, b.w), dx, dy, dz, r2, b.w, sr[k], acc, gacc);
                    }
                }
            } else {
                // FP64 (a pipe 1/64 of FP32): each lane first marks its in-support survivors,
                // then evaluates only those, so the evaluations follow the pairs in support
                unsigned msk = 0;
                for (int i = s, bit = 0; i < cnt; i += S, ++bit) {
                    const int k = (head + i) & (kPairList - 1);
                    const Q4 a = sA[k];
                    const T dx = xt[0] - a.x, dy = xt[1] - a.y, dz = xt[2] - a.z;
                    const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    if (r2 > T(0) && r2 < a.w && sI[k] != tgo) msk |= 1u << bit;
                }
                while (msk) {
                    const int bit = __ffs(msk) - 1;
                    msk &= msk - 1;
                    const int k = (head + s + bit * S) & (kPairList - 1);
                    const Q4 a = sA[k], b = sB[k];
                    const T dx = xt[0] - a.x, dy = xt[1] - a.y, dz = xt[2] - a.z;
                    const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    Pr::eval(ChebSeries<T>(tab, fits, r2, b.w), dx, dy, dz, r2, b.w, sr[k], acc, gacc);
                }
            }
            if constexpr (kTwo) {
#pragma unroll
                for (int j = 0; j < DU; ++j) two_float_acc(acc_hi[j], acc_lo[j], acc[j]);
#pragma unroll
                for (int j = 0; j < 3 * DU; ++j) two_float_acc(acc_hi[DU + j], acc_lo[DU + j], gacc[j]);
            } else {
#pragma unroll
                for (int j = 0; j < DU; ++j) acc_hi[j] += acc[j];
#pragma unroll
                for (int j = 0; j < 3 * DU; ++j) acc_hi[DU + j] += gacc[j];
            }
            head += cnt;
            __syncwarp();
        };
        const int e0 = doffs[li], e1 = doffs[li + 1];
        for (int e = e0; e < e1; ++e) {
            const DirectEntry de = dl[e];
            const int lev = de.code >> 6;
            const int sb[3] = {((de.code) & 3) - 1, ((de.code >> 2) & 3) - 1, ((de.code >> 4) & 3) - 1};
            chk |= lev == 0 && (sb[0] | sb[1] | sb[2]) != 0;
            // per-entry constants: nu^2 and 1/nu of the entry's level, image shift minus the
            // target leaf's centre
            T nu2, tinv;
            float Eh[3], El[3];
            double E[3];
            if constexpr (kTwo) {
                tinv = inv_s_f * pow2f(lev);
                nu2 = s2_f * pow2f(-2 * lev);
                for (int a = 0; a < 3; ++a) {
                    const float sh = sb[a] == 0 ? 0.f : (sb[a] > 0 ? Lh[a] : -Lh[a]);
                    const float sl = sb[a] == 0 ? 0.f : (sb[a] > 0 ? Ll[a] : -Ll[a]);
                    two_float_add(sh, sl, ch[a], cl[a], Eh[a], El[a]);
                }
            } else {
                tinv = (T)ldexp(inv_s, lev);
                nu2 = (T)ldexp(s2, -2 * lev);
                for (int a = 0; a < 3; ++a) E[a] = (double)sb[a] * g.L[a] - c[a];
            }
            const T lim = nu2 * box_margin;
            for (int base = de.start; base < de.end; base += 32) {
                const int si = base + lane;
                bool keep = false;
                Q4 a, b;
                if (si < de.end) {
                    if constexpr (kTwo) {
                        const float4* rp = out.pk + (int64_t)si * RQ;
                        const float4 p0 = rp[0], p1 = rp[1];
                        two_float_add(p0.x, p1.x, Eh[0], El[0], a.x, b.x);
                        two_float_add(p0.y, p1.y, Eh[1], El[1], a.y, b.y);
                        two_float_add(p0.z, p1.z, Eh[2], El[2], a.z, b.z);
                    } else {
                        a.x = (T)(xs[si] + E[0]);
                        a.y = (T)(xs[N + si] + E[1]);
                        a.z = (T)(xs[2 * N + si] + E[2]);
                        b.x = b.y = b.z = T(0);
                    }
                    const T px = a.x + b.x, py = a.y + b.y, pz = a.z + b.z;
                    const T gx = max(T(0), max(blo[0] - px, px - bhi[0]));
                    const T gy = max(T(0), max(blo[1] - py, py - bhi[1]));
                    const T gz = max(T(0), max(blo[2] - pz, pz - bhi[2]));
                    keep = fma(gx, gx, fma(gy, gy, gz * gz)) < lim;
                }
                const unsigned bal = __ballot_sync(full, keep);
                if (keep) {
                    const int slot = (tail + __popc(bal & below)) & (kPairList - 1);
                    a.w = nu2;
                    b.w = tinv;
                    sA[slot] = a;
                    sB[slot] = b;
                    sI[slot] = out.orig[si];
                    if constexpr (kTwo) {
                        const float4* rp = out.pk + (int64_t)si * RQ;
                        const float* rf = reinterpret_cast<const float*>(rp);
#pragma unroll
                        for (int a2 = 0; a2 < DR; ++a2) sr[slot][a2] = rf[point_record_rho(a2)];
                    } else {
#pragma unroll
                        for (int a2 = 0; a2 < DR; ++a2) sr[slot][a2] = (T)out.rs[(int64_t)si * DR + a2];
                    }
                }
                tail += __popc(bal);
                if (tail - head >= 32) run_block(32);
            }
        }
        if (tail > head) run_block(tail - head);
        // the S splits of a target, combined in a fixed order (every lane gets the same sum)
        double accd[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) accd[j] = (double)acc_hi[j] + (double)acc_lo[j];
        for (int o = m; o < 32; o <<= 1) {
#pragma unroll
            for (int j = 0; j < NA; ++j) accd[j] += __shfl_xor_sync(full, accd[j], o);
        }
        const int oi = out.perm[tg];
        if (s == 0 && oi < out.n_orig) {
            const double ks = KScale<K>::v;
#pragma unroll
            for (int j = 0; j < DU; ++j) out.pot[(int64_t)oi * DU + j] = ks * accd[j];
            if (GRAD && out.grad) {
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < DU; ++j) out.grad[((int64_t)oi * 3 + i) * DU + j] = ks * accd[DU + i * DU + j];
            }
        }
    }
}

template <class T, int DR>
inline size_t pair_smem() {
    return (size_t)kPairWarps * PairSmem<T, DR>::bytes;
}

constexpr int kLeafExpThreads = 128;

template <class T, int K, bool GRAD>
__global__ void __launch_bounds__(kLeafExpThreads) k_leafexp(int nleaf, const int* __restrict__ leaves, BoxArrays B,
                                                            Tab<T> tab, Geo g, const T* __restrict__ coef,
                                                            const double* __restrict__ xs, int64_t N, LeafOut out,
                                                            int direct_leaf) {
    using Pr = Pair<T, K, GRAD>;
    constexpr int DR = Pr::DR, DU = Pr::DU, MQ = kMaxPFast / 4;
    constexpr bool kTwo = sizeof(T) == 4;
    const int p = tab.p, p2 = p * p, p3 = p2 * p, PQ = (p + 3) & ~3, ng = PQ >> 2;
    extern __shared__ __align__(16) unsigned char dsme[];
    T* cs = reinterpret_cast<T*>(dsme);   // one output component's coefficients, rows padded to PQ
    const int tt = threadIdx.x;
    for (int li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const int box = leaves[li];
        const int l = B.level[box];
        const double r = ldexp(g.s, -l);                 // the leaf (self term)
        // the box whose expansion is evaluated: the leaf, or with direct_leaf its parent
        const int eb = (direct_leaf && l > 0) ? B.parent[box] : box;
        const int le = B.level[eb];
        const double re = ldexp(g.s, -le), half = 0.5 * re;
        const double c[3] = {(B.ix[3 * eb] + 0.5) * re, (B.ix[3 * eb + 1] + 0.5) * re, (B.ix[3 * eb + 2] + 0.5) * re};
        float ch[3], cl[3];
        for (int a = 0; a < 3; ++a) split_double(-c[a], ch[a], cl[a]);
        const int st = B.start[box], en = B.end[box];
        for (int t0 = st; t0 < en; t0 += kLeafExpThreads) {
            const bool act = tt < en - t0;
            const int tg = t0 + tt;
            T xi[3] = {0, 0, 0};
            if (act) {
                const T ih = (T)(1.0 / half);
                constexpr int RQ = point_record_floats(DR) / 4;
                float4 p0 = make_float4(0, 0, 0, 0), p1 = p0;
                if constexpr (kTwo) {
                    p0 = out.pk[(int64_t)tg * RQ];
                    p1 = out.pk[(int64_t)tg * RQ + 1];
                }
                const float ph[3] = {p0.x, p0.y, p0.z}, pl[3] = {p1.x, p1.y, p1.z};
                for (int a = 0; a < 3; ++a) {
                    T x0, x1 = 0;
                    if constexpr (kTwo) two_float_add(ph[a], pl[a], ch[a], cl[a], x0, x1);
                    else x0 = (T)(xs[a * N + tg] - c[a]);
                    const T v = (x0 + x1) * ih;
                    xi[a] = v > T(1) ? T(1) : (v < T(-1) ? T(-1) : v);
                }
            }
            T Tz[kMaxPFast], dTz[kMaxPFast];
            {
                T tm2 = 0, tm1 = 1, um2 = 0, um1 = 1;
#pragma unroll
                for (int n = 0; n < kMaxPFast; ++n) {
                    T tn, dn;
                    if (n == 0) { tn = 1; dn = 0; }
                    else if (n == 1) { tn = xi[2]; dn = 1; tm2 = 1; tm1 = xi[2]; um2 = 1; um1 = 2 * xi[2]; }
                    else {
                        tn = 2 * xi[2] * tm1 - tm2;
                        dn = (T)n * um1;
                        const T un = 2 * xi[2] * um1 - um2;
                        tm2 = tm1; tm1 = tn; um2 = um1; um1 = un;
                    }
                    Tz[n] = n < p ? tn : T(0);
                    dTz[n] = n < p ? dn : T(0);
                }
            }
            T ev[DU], eg[3 * DU];
#pragma unroll
            for (int j = 0; j < DU; ++j) {
                __syncthreads();
                const T* cj = coef + ((size_t)eb * DU + j) * p3;
                for (int e = tt; e < p2 * PQ; e += kLeafExpThreads) {
                    const int n12 = e / PQ, n3 = e - n12 * PQ;
                    cs[e] = n3 < p ? cj[n12 * p + n3] : T(0);
                }
                __syncthreads();
                T S = 0, Sx = 0, Sy = 0, Sz = 0;
                if (act) {
                    if (ng == 5)
                        cheb_eval<T, 5, false, GRAD>(cs, p, ng, Tz, dTz, xi, S, Sx, Sy, Sz);
                    else if (ng == 6)
                        cheb_eval<T, 6, false, GRAD>(cs, p, ng, Tz, dTz, xi, S, Sx, Sy, Sz);
                    else
                        cheb_eval<T, MQ, true, GRAD>(cs, p, ng, Tz, dTz, xi, S, Sx, Sy, Sz);
                }
                const T sc = (T)(1.0 / half);
                ev[j] = S;
                eg[0 * DU + j] = Sx * sc;
                eg[1 * DU + j] = Sy * sc;
                eg[2 * DU + j] = Sz * sc;
            }
            // expansion + residual sums (written by k_pair), minus the self term
            if (act && out.perm[tg] < out.n_orig) {
                const int oi = out.perm[tg];
                const double inv_nuT = 1.0 / r;
                const double* rt = out.rs + (int64_t)tg * DR;
#pragma unroll
                for (int j = 0; j < DU; ++j) {
                    double v = (double)ev[j] + out.pot[(int64_t)oi * DU + j] + (out.ucst ? out.ucst[j] : 0.0);
                    for (int a = 0; a < DR; ++a) v -= out.self_val[j * DR + a] * inv_nuT * rt[a];
                    out.pot[(int64_t)oi * DU + j] = v;
                }
                if (GRAD && out.grad) {
                    const double in3 = inv_nuT * inv_nuT * inv_nuT;
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < DU; ++j) {
                            const int64_t o = ((int64_t)oi * 3 + i) * DU + j;
                            double v = (double)eg[i * DU + j] + out.grad[o];
                            for (int a = 0; a < DR; ++a) v -= out.self_grad[(i * DU + j) * DR + a] * in3 * rt[a];
                            out.grad[o] = v;
                        }
                }
            }
        }
    }
}

// Work units of k_leafexp_parent: chunks of kLeafExpThreads targets of one item (a non-leaf box
// with leaf children: the targets of those children; a cube that is a leaf: its targets).
// cnt[item] = the item's chunk count, cnt[n_nl + n_root] = 0 (exclusive-scanned afterwards).
__global__ void k_item_chunks(int n_nl, const int* __restrict__ nl_box, int n_root, BoxArrays B,
                              int* __restrict__ cnt) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item > n_nl + n_root) return;
    int n = 0;
    if (item < n_nl) {
        const int eb = nl_box[item], c0 = B.child0[eb];
        for (int o = 0; o < 8; ++o)
            if (B.child0[c0 + o] < 0) n += B.end[c0 + o] - B.start[c0 + o];
    } else if (item < n_nl + n_root) {
        const int eb = item - n_nl;
        if (B.child0[eb] < 0) n = B.end[eb] - B.start[eb];
    }
    cnt[item] = (n + kLeafExpThreads - 1) / kLeafExpThreads;
}

// The leaf expansions with direct_leaf (Sec. 3.1.5): the targets of the leaf children of a
// non-leaf box evaluate that box's expansion (the same polynomial as the children's shifted
// expansions), the targets of a cube that is a leaf its own.  Work unit = a chunk of
// kLeafExpThreads targets of one such item (woff: exclusive prefix of the chunk counts, every
// lane a target but in an item's last chunk); the item's coefficients are staged once per
// component.  Component by component, the expansion and its gradient are added to the residual
// sums of k_pair and the self term of the target's own leaf (Sec. 2.4) subtracted, in FP64.
template <class T, int K, bool GRAD>
__global__ void __launch_bounds__(kLeafExpThreads) k_leafexp_parent(int n_nl, const int* __restrict__ nl_box,
                                                                   int n_root, const int* __restrict__ woff,
                                                                   BoxArrays B, Tab<T> tab, Geo g,
                                                                   const T* __restrict__ coef,
                                                                   const double* __restrict__ xs, int64_t N,
                                                                   LeafOut out) {
    using Pr = Pair<T, K, GRAD>;
    constexpr int DR = Pr::DR, DU = Pr::DU, MQ = kMaxPFast / 4;
    constexpr bool kTwo = sizeof(T) == 4;
    constexpr int RQ = point_record_floats(DR) / 4;
    const int p = tab.p, p2 = p * p, p3 = p2 * p, PQ = (p + 3) & ~3, ng = PQ >> 2;
    extern __shared__ __align__(16) unsigned char dsme[];
    T* cs = reinterpret_cast<T*>(dsme);   // one component's coefficients, rows padded to PQ
    __shared__ int rng[8][2];
    __shared__ int rpre[9];
    __shared__ int nrng;
    const int tt = threadIdx.x;
    const int n_items = n_nl + n_root, total = woff[n_items];
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        // the item of chunk w: the last with woff[item] <= w (woff[n_items] = total > w)
        int lo = 0, hi = n_items;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (woff[mid] <= w) lo = mid; else hi = mid;
        }
        const int item = lo, vbeg = (w - woff[item]) * kLeafExpThreads;
        int eb;
        __syncthreads();
        if (item < n_nl) {
            eb = nl_box[item];
            if (tt == 0) {
                int k = 0;
                const int c0 = B.child0[eb];
                for (int o = 0; o < 8; ++o)
                    if (B.child0[c0 + o] < 0) { rng[k][0] = B.start[c0 + o]; rng[k][1] = B.end[c0 + o]; ++k; }
                nrng = k;
            }
        } else {
            eb = item - n_nl;
            if (tt == 0) {
                nrng = (B.child0[eb] < 0) ? 1 : 0;
                rng[0][0] = B.start[eb];
                rng[0][1] = B.end[eb];
            }
        }
        __syncthreads();
        if (tt == 0) {
            rpre[0] = 0;
            for (int k = 0; k < nrng; ++k) rpre[k + 1] = rpre[k] + rng[k][1] - rng[k][0];
        }
        __syncthreads();
        const int nr = nrng, vend = min(rpre[nr], vbeg + kLeafExpThreads);
        const int le = B.level[eb];
        // the targets' own leaves: the children (level le + 1), or the cube itself
        const double rT = ldexp(g.s, -(item < n_nl ? le + 1 : le));
        const double re = ldexp(g.s, -le), half = 0.5 * re;
        const double c[3] = {(B.ix[3 * eb] + 0.5) * re, (B.ix[3 * eb + 1] + 0.5) * re, (B.ix[3 * eb + 2] + 0.5) * re};
        float ch[3], cl[3];
        for (int a = 0; a < 3; ++a) split_double(-c[a], ch[a], cl[a]);
        const T ih = (T)(1.0 / half);
        for (int j = 0; j < DU; ++j) {
            __syncthreads();
            const T* cj = coef + ((size_t)eb * DU + j) * p3;
            for (int e = tt; e < p2 * PQ; e += kLeafExpThreads) {
                const int n12 = e / PQ, n3 = e - n12 * PQ;
                cs[e] = n3 < p ? cj[n12 * p + n3] : T(0);
            }
            __syncthreads();
            {
                const int v = vbeg + tt;
                const bool act = v < vend;
                int tg = 0;
                if (act) {
                    int k = 0;
                    while (rpre[k + 1] <= v) ++k;
                    tg = rng[k][0] + (v - rpre[k]);
                }
                T xi[3] = {0, 0, 0};
                if (act) {
                    float4 p0 = make_float4(0, 0, 0, 0), p1 = p0;
                    if constexpr (kTwo) {
                        p0 = out.pk[(int64_t)tg * RQ];
                        p1 = out.pk[(int64_t)tg * RQ + 1];
                    }
                    const float ph[3] = {p0.x, p0.y, p0.z}, pl[3] = {p1.x, p1.y, p1.z};
                    for (int a = 0; a < 3; ++a) {
                        T x0, x1 = 0;
                        if constexpr (kTwo) two_float_add(ph[a], pl[a], ch[a], cl[a], x0, x1);
                        else x0 = (T)(xs[a * N + tg] - c[a]);
                        const T w = (x0 + x1) * ih;
                        xi[a] = w > T(1) ? T(1) : (w < T(-1) ? T(-1) : w);
                    }
                }
                T Tz[kMaxPFast], dTz[kMaxPFast];
                {
                    T tm2 = 0, tm1 = 1, um2 = 0, um1 = 1;
#pragma unroll
                    for (int n = 0; n < kMaxPFast; ++n) {
                        T tn, dn;
                        if (n == 0) { tn = 1; dn = 0; }
                        else if (n == 1) { tn = xi[2]; dn = 1; tm2 = 1; tm1 = xi[2]; um2 = 1; um1 = 2 * xi[2]; }
                        else {
                            tn = 2 * xi[2] * tm1 - tm2;
                            dn = (T)n * um1;
                            const T un = 2 * xi[2] * um1 - um2;
                            tm2 = tm1; tm1 = tn; um2 = um1; um1 = un;
                        }
                        Tz[n] = n < p ? tn : T(0);
                        dTz[n] = n < p ? dn : T(0);
                    }
                }
                T S = 0, Sx = 0, Sy = 0, Sz = 0;
                if (act) {
                    if (ng == 5)
                        cheb_eval<T, 5, false, GRAD>(cs, p, ng, Tz, dTz, xi, S, Sx, Sy, Sz);
                    else if (ng == 6)
                        cheb_eval<T, 6, false, GRAD>(cs, p, ng, Tz, dTz, xi, S, Sx, Sy, Sz);
                    else
                        cheb_eval<T, MQ, true, GRAD>(cs, p, ng, Tz, dTz, xi, S, Sx, Sy, Sz);
                }
                if (act && out.perm[tg] < out.n_orig) {
                    const int oi = out.perm[tg];
                    const double inv_nuT = 1.0 / rT;
                    const double* rt = out.rs + (int64_t)tg * DR;
                    double vv = (double)S + out.pot[(int64_t)oi * DU + j] + (out.ucst ? out.ucst[j] : 0.0);
                    for (int a = 0; a < DR; ++a) vv -= out.self_val[j * DR + a] * inv_nuT * rt[a];
                    out.pot[(int64_t)oi * DU + j] = vv;
                    if (GRAD && out.grad) {
                        const double in3 = inv_nuT * inv_nuT * inv_nuT;
                        const double sc = 1.0 / half;
                        const T gs[3] = {Sx, Sy, Sz};
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            const int64_t o = ((int64_t)oi * 3 + i) * DU + j;
                            double gv = (double)(gs[i] * (T)sc) + out.grad[o];
                            for (int a = 0; a < DR; ++a) gv -= out.self_grad[(i * DU + j) * DR + a] * in3 * rt[a];
                            out.grad[o] = gv;
                        }
                    }
                }
            }
        }
    }
}

template <class T>
inline size_t leafexp_smem(int p) {
    const int PQ = (p + 3) & ~3;
    return (size_t)p * p * PQ * sizeof(T);
}


}  // namespace dmk

namespace dmk {

// Upward pass child -> parent (Sec. 3.1.2) on thread-block clusters: cluster = parent box,
// CTA rank o = child octant.  Each CTA applies (I_o^T x I_o^T x I_o^T) to its child's proxy
// charges (three fiber contractions in shared memory), then the eight CTAs reduce the eight
// contributions through distributed shared memory in the fixed order o = 0..7, each CTA
// writing one eighth of the parent's tensor.
//   With direct_leaf (the leaf sources already anterpolated onto the parent grid, k_anterp3),
// leaf children contribute nothing here: a parent with only leaf children is skipped, and the
// non-leaf children's sum is added to the proxy when the parent has leaf children (stored
// otherwise).
template <class T, int MAXP>
__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__((MAXP * MAXP / 2 + 31) / 32 * 32, sizeof(T) == 4 ? 2 : 1)
    k_up_cluster(const int* __restrict__ nl_box, BoxArrays B, Tab<T> tab, T* __restrict__ proxy, int direct_leaf) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int o = (int)cl.block_rank();
    const int bi = blockIdx.x >> 3;
    const int p = tab.p, p2 = p * p, p3 = p2 * p, P = odd_pitch(p), drho = tab.d_rho;
    const int Pb0 = nl_box[bi], c00 = B.child0[Pb0];
    int n_leafc = 0;
    for (int q = 0; q < 8; ++q) n_leafc += B.child0[c00 + q] < 0;
    if (direct_leaf && n_leafc == 8) return;      // the same for every CTA of the cluster
    const bool skip_mine = direct_leaf && B.child0[c00 + o] < 0;
    const bool add = direct_leaf && n_leafc > 0;
    T* Mo = reinterpret_cast<T*>(dsmem);                 // 3 x MAXP x MAXP, one per axis
    T* bufA = Mo + 3 * MAXP * MAXP;
    T* bufB = bufA + p * p * P;
    for (int ax = 0; ax < 3; ++ax) {
        const int bit = (o >> ax) & 1;
        load_op<T, MAXP>(Mo + ax * MAXP * MAXP, p, [&](int k, int j) { return tab.Ioct[(bit * p + k) * p + j]; });
    }
    // fibers f and f + H of the p^2 fibers per thread
    const int H = (p2 + 1) / 2;
    const int f = threadIdx.x;
    const bool own = f < H, two = own && f + H < p2;
    const int fa0 = own ? f / p : 0, fb0 = own ? f % p : 0;
    const int fa1 = two ? (f + H) / p : 0, fb1 = two ? (f + H) % p : 0;
    const int Pb = nl_box[bi];
    const int C = B.child0[Pb] + o;
    const int lo = (o * p3) >> 3, hi = ((o + 1) * p3) >> 3;
    for (int a = 0; a < drho; ++a) {
        if (skip_mine) {
            // a leaf child: its sources are already in the parent's proxy
            for (int e = threadIdx.x; e < p3; e += blockDim.x) bufB[e] = T(0);
            cl.sync();
            T* out = proxy + ((size_t)Pb * drho + a) * p3;
            for (int e = lo + threadIdx.x; e < hi; e += blockDim.x) {
                T sum = 0;
#pragma unroll
                for (int r = 0; r < 8; ++r) sum += cl.map_shared_rank(bufB, r)[e];
                out[e] = add ? out[e] + sum : sum;
            }
            cl.sync();
            continue;
        }
        __syncthreads();
        load_padded_batched<T, MAXP>(bufA, proxy + ((size_t)C * drho + a) * p3, p, P);
        __syncthreads();
        T t0[MAXP], t1[MAXP];
        if (own) {
            fiber_contract2<T, MAXP>(bufA, p, P, 2, fa0, fb0, fa1, fb1, two, Mo + 2 * MAXP * MAXP, t0, t1);
            fiber_store<T, MAXP>(bufB, p, P, 2, fa0, fb0, t0);
            if (two) fiber_store<T, MAXP>(bufB, p, P, 2, fa1, fb1, t1);
        }
        __syncthreads();
        if (own) {
            fiber_contract2<T, MAXP>(bufB, p, P, 1, fa0, fb0, fa1, fb1, two, Mo + 1 * MAXP * MAXP, t0, t1);
            fiber_store<T, MAXP>(bufA, p, P, 1, fa0, fb0, t0);
            if (two) fiber_store<T, MAXP>(bufA, p, P, 1, fa1, fb1, t1);
        }
        __syncthreads();
        if (own) fiber_contract2<T, MAXP>(bufA, p, P, 0, fa0, fb0, fa1, fb1, two, Mo, t0, t1);
        // this child's contribution, unpadded, in bufB (free since the second contraction)
        if (own) {
#pragma unroll
            for (int j = 0; j < MAXP; ++j)
                if (j < p) {
                    bufB[(j * p + fa0) * p + fb0] = t0[j];
                    if (two) bufB[(j * p + fa1) * p + fb1] = t1[j];
                }
        }
        cl.sync();
        T* out = proxy + ((size_t)Pb * drho + a) * p3;
        for (int e = lo + threadIdx.x; e < hi; e += blockDim.x) {
            T sum = 0;
#pragma unroll
            for (int r = 0; r < 8; ++r) sum += cl.map_shared_rank(bufB, r)[e];
            out[e] = add ? out[e] + sum : sum;
        }
        cl.sync();
    }
}

// Shift to children (Sec. 3.1.4), one CTA per (parent, child octant): non-leaf child
// local += (I_o x I_o x I_o) parent; leaf child local += (A_o x A_o x A_o) parent, A_o = C I_o,
// the Chebyshev coefficients of the child's interpolant.
//   With direct_leaf the leaf children are skipped: their targets evaluate the parent's
// expansion (k_box_coef, k_leafexp), the same polynomial.
template <class T, int MAXP>
__global__ void __launch_bounds__((MAXP * MAXP + 31) / 32 * 32, sizeof(T) == 4 ? 2 : 1) k_shift_child(const int* __restrict__ nl_box, BoxArrays B, Tab<T> tab,
                                                     T* __restrict__ local, int direct_leaf) {
    const int o = blockIdx.x & 7;
    const int bi = blockIdx.x >> 3;
    const int p = tab.p, p2 = p * p, p3 = p2 * p, P = odd_pitch(p), du = tab.d_u;
    T* Mo = reinterpret_cast<T*>(dsmem);                 // 3 x MAXP x MAXP, rows k = parent index
    T* bufA = Mo + 3 * MAXP * MAXP;
    T* bufB = bufA + p * p * P;
    const int Pb = nl_box[bi];
    const int C = B.child0[Pb] + o;
    const bool leaf_child = B.child0[C] < 0;
    if (direct_leaf && leaf_child) return;
    const T* src = leaf_child ? tab.Aoct : tab.Ioct;
    for (int ax = 0; ax < 3; ++ax) {
        const int bit = (o >> ax) & 1;
        load_op<T, MAXP>(Mo + ax * MAXP * MAXP, p, [&](int k, int j) { return src[(bit * p + j) * p + k]; });
    }
    const int f = threadIdx.x;
    const bool own = f < p2;
    const int fa = own ? f / p : 0, fb = own ? f % p : 0;
    for (int j = 0; j < du; ++j) {
        __syncthreads();
        load_padded_batched<T, MAXP>(bufA, local + ((size_t)Pb * du + j) * p3, p, P);
        __syncthreads();
        T t[MAXP];
        if (own) {
            fiber_contract<T, MAXP>(bufA, p, P, 2, fa, fb, Mo + 2 * MAXP * MAXP, t);
            fiber_store<T, MAXP>(bufB, p, P, 2, fa, fb, t);
        }
        __syncthreads();
        if (own) {
            fiber_contract<T, MAXP>(bufB, p, P, 1, fa, fb, Mo + 1 * MAXP * MAXP, t);
            fiber_store<T, MAXP>(bufA, p, P, 1, fa, fb, t);
        }
        __syncthreads();
        if (own) {
            fiber_contract<T, MAXP>(bufA, p, P, 0, fa, fb, Mo, t);
            T* out = local + ((size_t)C * du + j) * p3;
            if (leaf_child) {                          // only the shift writes a leaf's expansion
#pragma unroll
                for (int jj = 0; jj < MAXP; ++jj)
                    if (jj < p) out[(jj * p + fa) * p + fb] = t[jj];
            } else {                                   // non-leaf: add to its plane-wave part
#pragma unroll
                for (int jj = 0; jj < MAXP; ++jj)
                    if (jj < p) out[(jj * p + fa) * p + fb] += t[jj];
            }
        }
    }
}


// Grid values -> Chebyshev coefficients in place (c = (C x C x C) u, Sec. 3.1.5), one CTA per
// non-leaf box that has a leaf child: those children's targets evaluate the parent's expansion.
template <class T, int MAXP>
__global__ void __launch_bounds__((MAXP * MAXP + 31) / 32 * 32, sizeof(T) == 4 ? 2 : 1)
    k_box_coef(const int* __restrict__ nl_box, BoxArrays B, Tab<T> tab, T* __restrict__ local) {
    const int p = tab.p, p2 = p * p, p3 = p2 * p, P = odd_pitch(p), du = tab.d_u;
    const int Pb = nl_box[blockIdx.x];
    const int c0 = B.child0[Pb];
    bool any_leaf = false;
    for (int q = 0; q < 8; ++q) any_leaf = any_leaf || B.child0[c0 + q] < 0;
    if (!any_leaf) return;
    T* Mo = reinterpret_cast<T*>(dsmem);                 // MAXP x MAXP: Mo[k][n] = C[n][k]
    T* bufA = Mo + MAXP * MAXP;
    T* bufB = bufA + p * p * P;
    load_op<T, MAXP>(Mo, p, [&](int k, int j) { return tab.Cm[j * p + k]; });
    const int f = threadIdx.x;
    const bool own = f < p2;
    const int fa = own ? f / p : 0, fb = own ? f % p : 0;
    for (int j = 0; j < du; ++j) {
        T* u = local + ((size_t)Pb * du + j) * p3;
        __syncthreads();
        load_padded_batched<T, MAXP>(bufA, u, p, P);
        __syncthreads();
        T t[MAXP];
        if (own) {
            fiber_contract<T, MAXP>(bufA, p, P, 2, fa, fb, Mo, t);
            fiber_store<T, MAXP>(bufB, p, P, 2, fa, fb, t);
        }
        __syncthreads();
        if (own) {
            fiber_contract<T, MAXP>(bufB, p, P, 1, fa, fb, Mo, t);
            fiber_store<T, MAXP>(bufA, p, P, 1, fa, fb, t);
        }
        __syncthreads();
        if (own) {
            fiber_contract<T, MAXP>(bufA, p, P, 0, fa, fb, Mo, t);
#pragma unroll
            for (int jj = 0; jj < MAXP; ++jj)
                if (jj < p) u[(jj * p + fa) * p + fb] = t[jj];
        }
    }
}
}  // namespace dmk
