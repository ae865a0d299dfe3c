// Device-side helpers: complex arithmetic, Morton keys, table views, precision traits.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dmk {

template <class T> struct Cx { T x, y; };
template <class T> __host__ __device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T> __host__ __device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T> __host__ __device__ __forceinline__ Cx<T> cconj(Cx<T> a) { return {a.x, -a.y}; }
// a += b * c
template <class T> __device__ __forceinline__ void cfma(Cx<T>& a, Cx<T> b, Cx<T> c) {
    a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
// a += b * real
template <class T> __device__ __forceinline__ void cfmar(Cx<T>& a, Cx<T> b, T r) {
    a.x = fma(b.x, r, a.x);
    a.y = fma(b.y, r, a.y);
}

// ---- keys: cell key at level l = (cube << 3l) | interleave(px, py, pz) with x the lowest bit
__host__ __device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ULL;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ULL;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00fULL;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffULL;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffULL;
    x = (x ^ (x >> 32)) & 0x1fffffULL;
    return (uint32_t)x;
}

// Geometry of the cube tiling.  Coordinates inside the library are taken relative to the lower
// corner of Omega_ext (origin; nonzero only on padded axes), so boxes start at 0.
struct Geo {
    double L[3];       // the periods (true lengths)
    double s;          // cube side
    int M[3];          // cubes per axis, padding included
    int periodic[3];   // the forest wraps along the axis
    int wrap[3];       // input coordinates are wrapped mod L along the axis (axes < D)
    double origin[3];
    int padded[3];
    int D;
    // 1/s and 1/L_i where they are powers of two (division by them is then exactly the
    // multiplication, bit for bit), else 0: the quantisation and the wrap use the division
    double inv_s_pow2;
    double inv_L_pow2[3];
};

// global integer index of a cell -> key (valid indices only)
__host__ __device__ __forceinline__ uint64_t cell_key(const Geo& g, int level, const int ix[3]) {
    uint32_t m[3], p[3];
    for (int i = 0; i < 3; ++i) {
        m[i] = (uint32_t)ix[i] >> level;
        p[i] = (uint32_t)ix[i] & ((1u << level) - 1u);
    }
    uint64_t cube = m[0] + (uint64_t)g.M[0] * (m[1] + (uint64_t)g.M[1] * m[2]);
    uint64_t morton = spread3(p[0]) | (spread3(p[1]) << 1) | (spread3(p[2]) << 2);
    return (cube << (3 * level)) | morton;
}
__host__ __device__ __forceinline__ void cell_ix(const Geo& g, int level, uint64_t key, int ix[3]) {
    uint64_t cube = key >> (3 * level);
    uint64_t morton = key & ((level == 0) ? 0ULL : ((1ULL << (3 * level)) - 1ULL));
    int m0 = (int)(cube % g.M[0]);
    int m1 = (int)((cube / g.M[0]) % g.M[1]);
    int m2 = (int)(cube / ((uint64_t)g.M[0] * g.M[1]));
    ix[0] = (m0 << level) | (int)compact3(morton);
    ix[1] = (m1 << level) | (int)compact3(morton >> 1);
    ix[2] = (m2 << level) | (int)compact3(morton >> 2);
}

// neighbour of ix at level by offset d; returns false if outside a free axis.  shift[i] counts
// whole periods (-1, 0, 1) so that the image sits at (wrapped neighbour) + shift * L.
__host__ __device__ __forceinline__ bool neighbour(const Geo& g, int level, const int ix[3], const int d[3],
                                                   int out[3], int shift[3]) {
    for (int i = 0; i < 3; ++i) {
        int n = g.M[i] << level;
        int v = ix[i] + d[i];
        shift[i] = 0;
        if (v < 0 || v >= n) {
            if (!g.periodic[i]) return false;
            if (v < 0) { v += n; shift[i] = -1; } else { v -= n; shift[i] = 1; }
        }
        out[i] = v;
    }
    return true;
}

// view of the per-precision tables on the device
template <class T> struct Tab {
    int p, nf, NF, nfh, d_rho, d_u, kernel, level_power;
    const T* nodes;
    const T* bary;
    const T* Ioct;       // 2 x p x p
    const T* Aoct;       // 2 x p x p: parent grid -> child Chebyshev coefficients
    const T* Cm;         // p x p
    const Cx<T>* E;      // NF x p
    const T* gdiff;      // NF x NF x nfh
    const T* fit;        // concatenated Chebyshev series
    int off_q, n_q, off_f, n_f, off_g, n_g, off_dq, n_dq, off_df, n_df, off_dg, n_dg;
    const float* herm;   // FP32 path: piecewise cubic tables of the six series (see HermSeries)
};

// four values loaded as one vector from shared memory
template <class T>
struct alignas(4 * sizeof(T)) Quad {
    T x, y, z, w;
};

// Clenshaw evaluation of sum_k a_k T_k(t)
template <class T> __device__ __forceinline__ T clenshaw(const T* a, int n, T t) {
    T b1 = 0, b2 = 0;
    T t2 = t + t;
    for (int k = n - 1; k >= 1; --k) {
        T b0 = fma(t2, b1, a[k] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fma(t, b1, a[0] - b2);
}

// ---- residual series (App. B, "precomputed polynomial approximations"): q, f, g and their
// s-derivatives as functions of s = r^2 / nu^2 in [0, 1] ------------------------------------
enum { kSerQ = 0, kSerF, kSerG, kSerDQ, kSerDF, kSerDG };

// Chebyshev series in t = 2 s - 1, coefficients at the offsets of Tab (FP64 path and p > kMaxPFast)
template <class T>
struct ChebSeries {
    const Tab<T>& tb;
    const T* fit;
    T t;
    __device__ __forceinline__ ChebSeries(const Tab<T>& tb_, const T* fit_, T r2, T inv_nu)
        : tb(tb_), fit(fit_), t(fma(T(2) * r2, inv_nu * inv_nu, T(-1))) {}
    __device__ __forceinline__ T operator()(int k) const {
        switch (k) {
            case kSerQ: return clenshaw(fit + tb.off_q, tb.n_q, t);
            case kSerF: return clenshaw(fit + tb.off_f, tb.n_f, t);
            case kSerG: return clenshaw(fit + tb.off_g, tb.n_g, t);
            case kSerDQ: return clenshaw(fit + tb.off_dq, tb.n_dq, t);
            case kSerDF: return clenshaw(fit + tb.off_df, tb.n_df, t);
            default: return clenshaw(fit + tb.off_dg, tb.n_dg, t);
        }
    }
};

// Piecewise cubic Hermite form of the same series for the FP32 path: kHermNT intervals of s, the
// interval i holding (c0, c1, c2, c3) with X = c0 + u (c1 + u (c2 + u c3)), u = s kHermNT - i,
// built on the host from the FP64 series values and derivatives at the interval ends.  Table
// k (series order above) starts at tbl + k kHermNT.
constexpr int kHermNT = 256;

// 2^n exactly, from the exponent bits (|n| well inside the normal range): no FP64 or
// conversion instruction
__device__ __forceinline__ float pow2f(int n) { return __int_as_float((n + 127) << 23); }
__device__ __forceinline__ double pow2d(int n) { return __longlong_as_double((long long)(n + 1023) << 52); }
template <class T> __device__ __forceinline__ T pow2t(int n);
template <> __device__ __forceinline__ float pow2t<float>(int n) { return pow2f(n); }
template <> __device__ __forceinline__ double pow2t<double>(int n) { return pow2d(n); }

struct HermSeries {
    const Quad<float>* tbl;
    int i;
    float u;
    __device__ __forceinline__ HermSeries(const Quad<float>* tbl_, float r2, float inv_nu) : tbl(tbl_) {
        const float x = r2 * (inv_nu * inv_nu) * (float)kHermNT;       // in [0, kHermNT]
        // floor(x) without a float-to-integer conversion: with round-down, 1.5 2^23 + x keeps
        // floor(x) in its low mantissa bits (0 <= x < 2^22); the FP32 additions are exact
        const float big = 12582912.0f;
        const float y = __fadd_rd(x, big);
        i = min(__float_as_int(y) - __float_as_int(big), kHermNT - 1);
        u = x - fminf(y - big, (float)(kHermNT - 1));
    }
    __device__ __forceinline__ float operator()(int k) const {
        const Quad<float> c = tbl[k * kHermNT + i];
        return fmaf(u, fmaf(u, fmaf(u, c.w, c.z), c.y), c.x);
    }
};

}  // namespace dmk
