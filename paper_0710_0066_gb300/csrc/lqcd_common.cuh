// lqcd_common.cuh -- internal types and device helpers of the GB300 library.
//
// Internal field layouts (structure of arrays, one parity block after the
// other, so that a warp reads 128-bit words of consecutive sites):
//   double spinor  [parity][12 complex][Vh]   double2
//   single spinor  [parity][6][Vh]            float4  (two complex each)
//   half spinor    [parity][3][Vh]            uint4   (four complex each)
//                  + [parity][Vh] float scale (max |component| of the site)
//   bf16 spinor    [parity][3][Vh]            uint4   (four complex each, no scale)
//   double gauge   [mu][parity][9][Vh]        double2 (full 3x3)
//   single gauge   [mu][parity][3][Vh]        float4  (rows 0 and 1)
//   half gauge     [mu][parity][3][Vh]        uint2   (rows 0 and 1)
//   bf16 gauge     the same, following the half gauge in one allocation
// Row 2 of a compressed link is rebuilt as conj(row0 x row1) (SU(3)).
// eo index of a site: lexicographic index / 2 (L3 is even).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lqcd.h"

#define LQ_HD __host__ __device__ __forceinline__

#include "lqcd_df.cuh"

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
struct Geo {
    int L[4];
    int V, Vh, V3;
    int l0, nb, bc_t;
    int Sh;   // sites of one parity in one slab = l0 * V3 / 2
    int l0s;  // iterated decomposition: sub-slab thickness l0 / 2, or 0
    // index helpers set by geo_finish: log2 of L1, L2, L3 when all three are
    // powers of two (lg[0] = 1), and bit t of face / sface set when slice t
    // starts a slab / sub-slab (used when L0 <= 64)
    int lg[4];
    unsigned long long face, sface;
};

// fills the index helpers of g from L, l0 and l0s
inline void geo_finish(Geo& g)
{
    int ok = 1;
    for (int mu = 1; mu < 4; ++mu) {
        int k = 0;
        while ((1 << k) < g.L[mu]) ++k;
        g.lg[mu] = k;
        if ((1 << k) != g.L[mu]) ok = 0;
    }
    g.lg[0] = ok;
    g.face = g.sface = 0ull;
    if (g.L[0] <= 64)
        for (int t = 0; t < g.L[0]; ++t) {
            if (g.l0 > 0 && t % g.l0 == 0) g.face |= 1ull << t;
            if (g.l0s > 0 && t % g.l0s == 0) g.sface |= 1ull << t;
        }
}

// Geometry of the second level of the iterated decomposition (Sec. 1): the
// sub-slabs of thickness l0s play the part of the slabs, so every block
// kernel run on it works on W2 instead of W1.
inline Geo sub_geo(const Geo& g)
{
    Geo s = g;
    s.l0 = g.l0s;
    s.nb = g.L[0] / g.l0s;
    s.Sh = g.l0s * g.V3 / 2;
    s.l0s = 0;
    geo_finish(s);
    return s;
}

// coordinates of eo index i of parity p
LQ_HD void eo_coords(const Geo& g, int p, int i, int x[4])
{
    const int j = 2 * i;
    if (g.lg[0]) {  // L1, L2, L3 powers of two: shifts and masks
        x[3] = j & (g.L[3] - 1);
        int t = j >> g.lg[3];
        x[2] = t & (g.L[2] - 1);
        t >>= g.lg[2];
        x[1] = t & (g.L[1] - 1);
        x[0] = t >> g.lg[1];
    } else {
        x[3] = j % g.L[3];
        int t = j / g.L[3];
        x[2] = t % g.L[2];
        t /= g.L[2];
        x[1] = t % g.L[1];
        x[0] = t / g.L[1];
    }
    x[3] += (x[0] + x[1] + x[2] + x[3] + p) & 1;
}

LQ_HD int lex_of(const Geo& g, const int x[4])
{
    return ((x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
}

// ---------------------------------------------------------------------------
// complex arithmetic
// ---------------------------------------------------------------------------
template <class T>
struct cx {
    T re, im;
};
template <class T>
LQ_HD cx<T> mk(T a, T b) { return cx<T>{a, b}; }
template <class T>
LQ_HD cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T>
LQ_HD cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T>
LQ_HD cx<T> operator-(cx<T> a) { return {-a.re, -a.im}; }
template <class T>
LQ_HD cx<T> operator*(cx<T> a, cx<T> b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
template <class T>
LQ_HD cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <class T>
LQ_HD cx<T> conjx(cx<T> a) { return {a.re, -a.im}; }
template <class T>
LQ_HD cx<T> mul_i(cx<T> a) { return {-a.im, a.re}; }   // i a
template <class T>
LQ_HD cx<T> mul_mi(cx<T> a) { return {a.im, -a.re}; }  // -i a
// a^* b
template <class T>
LQ_HD cx<T> cjmul(cx<T> a, cx<T> b) { return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re}; }

template <class T>
struct Spinor {
    cx<T> c[4][3];
};
template <class T>
struct HalfSp {
    cx<T> c[2][3];
};
template <class T>
struct Su3 {
    cx<T> m[3][3];
};

template <class T>
LQ_HD void complete_row2(Su3<T>& u)
{
    u.m[2][0] = conjx(u.m[0][1] * u.m[1][2] - u.m[0][2] * u.m[1][1]);
    u.m[2][1] = conjx(u.m[0][2] * u.m[1][0] - u.m[0][0] * u.m[1][2]);
    u.m[2][2] = conjx(u.m[0][0] * u.m[1][1] - u.m[0][1] * u.m[1][0]);
}

// w = u v  /  w = u^dag v  on the two spin rows of a half spinor
template <class T>
LQ_HD void su3_mul_half(const Su3<T>& u, const HalfSp<T>& h, HalfSp<T>& w)
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            w.c[s][i] = u.m[i][0] * h.c[s][0] + u.m[i][1] * h.c[s][1] + u.m[i][2] * h.c[s][2];
}
template <class T>
LQ_HD void su3_dagmul_half(const Su3<T>& u, const HalfSp<T>& h, HalfSp<T>& w)
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            w.c[s][i] = cjmul(u.m[0][i], h.c[s][0]) + cjmul(u.m[1][i], h.c[s][1]) +
                        cjmul(u.m[2][i], h.c[s][2]);
}

// ---------------------------------------------------------------------------
// spin projection in the chiral basis (gamma_0 = [[0,-1],[-1,0]],
// gamma_k = [[0,-i s_k],[i s_k,0]]).  (1 + sg*gamma_mu) psi has rank 2:
//   upper half h = u + sg*Q_mu d, lower half = K_mu h,
// u = (psi0, psi1), d = (psi2, psi3).  sg = -1 gives (1 - gamma_mu).
// ---------------------------------------------------------------------------
// the same projection for one colour: (h0, h1) from the spin components
// (p0, p1, p2, p3) (the double-float sweep projects as its loads arrive)
template <class T>
LQ_HD void project1(int mu, int sg, const cx<T>& p0, const cx<T>& p1, const cx<T>& p2, const cx<T>& p3, cx<T>& h0,
                    cx<T>& h1)
{
    cx<T> a, b;
    switch (mu) {
        case 0: a = p2; b = p3; break;                  // gamma_0 psi = (-d, -u): h = u - sg d
        case 1: a = mul_i(p3); b = mul_i(p2); break;    // -i s1 d = (-i d1, -i d0): h = u - sg i s1 d
        case 2: a = p3; b = -p2; break;                 // i s2 d = (d1, -d0)
        default: a = mul_i(p2); b = mul_mi(p3); break;  // i s3 d = (i d0, -i d1)
    }
    if (sg < 0) { h0 = p0 + a; h1 = p1 + b; }
    else        { h0 = p0 - a; h1 = p1 - b; }
}

// colour i of acc += (1 + sg*gamma_mu) psi rebuilt from its upper half
// (w0, w1): lower half = sg * l with l = -w (mu = 0) or l = (i s_k) w (mu = k)
template <class T>
LQ_HD void accum_recon1(int mu, int sg, const cx<T>& w0, const cx<T>& w1, Spinor<T>& acc, int i)
{
    acc.c[0][i] = acc.c[0][i] + w0;
    acc.c[1][i] = acc.c[1][i] + w1;
    cx<T> l0, l1;
    switch (mu) {
        case 0: l0 = -w0; l1 = -w1; break;
        case 1: l0 = mul_i(w1); l1 = mul_i(w0); break;
        case 2: l0 = w1; l1 = -w0; break;
        default: l0 = mul_i(w0); l1 = mul_mi(w1); break;
    }
    if (sg < 0) { acc.c[2][i] = acc.c[2][i] - l0; acc.c[3][i] = acc.c[3][i] - l1; }
    else        { acc.c[2][i] = acc.c[2][i] + l0; acc.c[3][i] = acc.c[3][i] + l1; }
}

template <class T>
LQ_HD void project(int mu, int sg, const Spinor<T>& p, HalfSp<T>& h)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        cx<T> a, b;
        switch (mu) {
            case 0:  // gamma_0 psi = (-d, -u): h = u - sg d
                a = p.c[2][i]; b = p.c[3][i];
                if (sg < 0) { h.c[0][i] = p.c[0][i] + a; h.c[1][i] = p.c[1][i] + b; }
                else        { h.c[0][i] = p.c[0][i] - a; h.c[1][i] = p.c[1][i] - b; }
                break;
            case 1:  // gamma_1 psi upper = -i s1 d = (-i d1, -i d0): h = u - sg i s1 d
                a = mul_i(p.c[3][i]); b = mul_i(p.c[2][i]);
                if (sg < 0) { h.c[0][i] = p.c[0][i] + a; h.c[1][i] = p.c[1][i] + b; }
                else        { h.c[0][i] = p.c[0][i] - a; h.c[1][i] = p.c[1][i] - b; }
                break;
            case 2:  // i s2 d = (d1, -d0)
                a = p.c[3][i]; b = -p.c[2][i];
                if (sg < 0) { h.c[0][i] = p.c[0][i] + a; h.c[1][i] = p.c[1][i] + b; }
                else        { h.c[0][i] = p.c[0][i] - a; h.c[1][i] = p.c[1][i] - b; }
                break;
            default:  // i s3 d = (i d0, -i d1)
                a = mul_i(p.c[2][i]); b = mul_mi(p.c[3][i]);
                if (sg < 0) { h.c[0][i] = p.c[0][i] + a; h.c[1][i] = p.c[1][i] + b; }
                else        { h.c[0][i] = p.c[0][i] - a; h.c[1][i] = p.c[1][i] - b; }
                break;
        }
    }
}

// acc += (1 + sg*gamma_mu) psi rebuilt from its upper half w:
//   lower half = sg * l with l = -w (mu = 0) or l = (i s_k) w (mu = k)
template <class T>
LQ_HD void accum_recon(int mu, int sg, const HalfSp<T>& w, Spinor<T>& acc)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        acc.c[0][i] = acc.c[0][i] + w.c[0][i];
        acc.c[1][i] = acc.c[1][i] + w.c[1][i];
        cx<T> l0, l1;
        switch (mu) {
            case 0: l0 = -w.c[0][i]; l1 = -w.c[1][i]; break;
            case 1: l0 = mul_i(w.c[1][i]); l1 = mul_i(w.c[0][i]); break;
            case 2: l0 = w.c[1][i]; l1 = -w.c[0][i]; break;
            default: l0 = mul_i(w.c[0][i]); l1 = mul_mi(w.c[1][i]); break;
        }
        if (sg < 0) { acc.c[2][i] = acc.c[2][i] - l0; acc.c[3][i] = acc.c[3][i] - l1; }
        else        { acc.c[2][i] = acc.c[2][i] + l0; acc.c[3][i] = acc.c[3][i] + l1; }
    }
}

// ---------------------------------------------------------------------------
// field views
// ---------------------------------------------------------------------------
// PRECDF: double storage (fields and links), double-float arithmetic; the
// double sweeps of the mixed-precision path.  PRECDS: the same arithmetic
// on a spinor stored as df pairs (float4 = re.hi, im.hi, re.lo, im.lo per
// complex, 16 bytes like a double2), for intermediates that never leave
// the solver.  Internal, not API precisions.
// PRECBF: bfloat16 storage (FP32 arithmetic), no per-site scale.  The
// four storage precisions have the ids of the C-ABI's LQCD_PREC_*.
enum { PREC64 = 0, PREC32 = 1, PREC16 = 2, PRECBF = 3, PRECDF = 4, PRECDS = 5 };
constexpr int NPREC = 4;

struct SpinorF {  // one parity block of a spinor field in some precision
    void* v;      // double2* / float4* / uint4*
    float* nrm;   // half only
    int N;        // stride (sites of the parity block)
};

struct GaugeF {  // gauge field in some precision, [mu][parity][...][Vh]
    const void* v;
    int Vh;
};

template <int P>
struct Real;
template <>
struct Real<PREC64> {
    typedef double T;
};
template <>
struct Real<PREC32> {
    typedef float T;
};
template <>
struct Real<PREC16> {
    typedef float T;
};
template <>
struct Real<PRECBF> {
    typedef float T;
};
template <>
struct Real<PRECDF> {
    typedef df T;
};
template <>
struct Real<PRECDS> {
    typedef df T;
};

// RO = true: the field is not written during the kernel (read-only path);
// RO = false: plain coherent loads (fields updated inside a persistent kernel)
template <class V, bool RO>
__device__ __forceinline__ V ldv(const V* p)
{
    if (RO) return __ldg(p);
    return *p;
}

template <int P, bool RO>
struct SpIO;

template <bool RO>
struct SpIO<PREC64, RO> {
    static __device__ __forceinline__ void load(const SpinorF& f, int i, Spinor<double>& s)
    {
        const double2* p = (const double2*)f.v;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 d = ldv<double2, RO>(p + (size_t)c * f.N + i);
            s.c[c / 3][c % 3] = mk(d.x, d.y);
        }
    }
    static __device__ __forceinline__ void store(const SpinorF& f, int i, const Spinor<double>& s)
    {
        double2* p = (double2*)f.v;
#pragma unroll
        for (int c = 0; c < 12; ++c)
            p[(size_t)c * f.N + i] = make_double2(s.c[c / 3][c % 3].re, s.c[c / 3][c % 3].im);
    }
};

template <bool RO>
struct SpIO<PREC32, RO> {
    static __device__ __forceinline__ void load(const SpinorF& f, int i, Spinor<float>& s)
    {
        const float4* p = (const float4*)f.v;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 d = ldv<float4, RO>(p + (size_t)k * f.N + i);
            s.c[(2 * k) / 3][(2 * k) % 3] = mk(d.x, d.y);
            s.c[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(d.z, d.w);
        }
    }
    static __device__ __forceinline__ void store(const SpinorF& f, int i, const Spinor<float>& s)
    {
        float4* p = (float4*)f.v;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const cx<float> a = s.c[(2 * k) / 3][(2 * k) % 3];
            const cx<float> b = s.c[(2 * k + 1) / 3][(2 * k + 1) % 3];
            p[(size_t)k * f.N + i] = make_float4(a.re, a.im, b.re, b.im);
        }
    }
};

template <bool RO>
struct SpIO<PREC16, RO> {
    static __device__ __forceinline__ void load(const SpinorF& f, int i, Spinor<float>& s)
    {
        const uint4* p = (const uint4*)f.v;
        const float sc = ldv<float, RO>(f.nrm + i);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 d = ldv<uint4, RO>(p + (size_t)k * f.N + i);
            unsigned w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 v = __half22float2(*reinterpret_cast<__half2*>(&w[q]));
                const int c = 4 * k + q;
                s.c[c / 3][c % 3] = mk(v.x * sc, v.y * sc);
            }
        }
    }
    static __device__ __forceinline__ void store(const SpinorF& f, int i, const Spinor<float>& s)
    {
        float mx = 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c)
            mx = fmaxf(mx, fmaxf(fabsf(s.c[c / 3][c % 3].re), fabsf(s.c[c / 3][c % 3].im)));
        const float inv = mx > 0.f ? 1.0f / mx : 0.f;
        uint4* p = (uint4*)f.v;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            unsigned w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 4 * k + q;
                __half2 hv = __floats2half2_rn(s.c[c / 3][c % 3].re * inv, s.c[c / 3][c % 3].im * inv);
                w[q] = *reinterpret_cast<unsigned*>(&hv);
            }
            p[(size_t)k * f.N + i] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        f.nrm[i] = mx;
    }
};

template <bool RO>
struct SpIO<PRECBF, RO> {
    static __device__ __forceinline__ void load(const SpinorF& f, int i, Spinor<float>& s)
    {
        const uint4* p = (const uint4*)f.v;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 d = ldv<uint4, RO>(p + (size_t)k * f.N + i);
            unsigned w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 v = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w[q]));
                const int c = 4 * k + q;
                s.c[c / 3][c % 3] = mk(v.x, v.y);
            }
        }
    }
    static __device__ __forceinline__ void store(const SpinorF& f, int i, const Spinor<float>& s)
    {
        uint4* p = (uint4*)f.v;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            unsigned w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 4 * k + q;
                __nv_bfloat162 hv = __floats2bfloat162_rn(s.c[c / 3][c % 3].re, s.c[c / 3][c % 3].im);
                w[q] = *reinterpret_cast<unsigned*>(&hv);
            }
            p[(size_t)k * f.N + i] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
};

template <bool RO>
struct SpIO<PRECDF, RO> {
    static __device__ __forceinline__ void load(const SpinorF& f, int i, Spinor<df>& s)
    {
        const double2* p = (const double2*)f.v;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 d = ldv<double2, RO>(p + (size_t)c * f.N + i);
            s.c[c / 3][c % 3] = mk(df_split(d.x), df_split(d.y));
        }
    }
    static __device__ __forceinline__ void store(const SpinorF& f, int i, const Spinor<df>& s)
    {
        double2* p = (double2*)f.v;
#pragma unroll
        for (int c = 0; c < 12; ++c)
            p[(size_t)c * f.N + i] = make_double2(df_to_double(s.c[c / 3][c % 3].re), df_to_double(s.c[c / 3][c % 3].im));
    }
};

template <bool RO>
struct SpIO<PRECDS, RO> {
    static __device__ __forceinline__ void load(const SpinorF& f, int i, Spinor<df>& s)
    {
        const float4* p = (const float4*)f.v;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            float4 d = ldv<float4, RO>(p + (size_t)c * f.N + i);
            s.c[c / 3][c % 3] = mk(df(d.x, d.z), df(d.y, d.w));
        }
    }
    static __device__ __forceinline__ void store(const SpinorF& f, int i, const Spinor<df>& s)
    {
        float4* p = (float4*)f.v;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const cx<df> v = s.c[c / 3][c % 3];
            p[(size_t)c * f.N + i] = make_float4(v.re.hi, v.im.hi, v.re.lo, v.im.lo);
        }
    }
};

// a spinor of any arithmetic type as doubles
LQ_HD void to_double(const Spinor<double>& s, Spinor<double>& d) { d = s; }
LQ_HD void to_double(const Spinor<df>& s, Spinor<double>& d)
{
#pragma unroll
    for (int k = 0; k < 12; ++k)
        d.c[k / 3][k % 3] = mk(df_to_double(s.c[k / 3][k % 3].re), df_to_double(s.c[k / 3][k % 3].im));
}

template <int P, bool RO = true>
__device__ __forceinline__ void load_spinor(const SpinorF& f, int i, Spinor<typename Real<P>::T>& s)
{
    SpIO<P, RO>::load(f, i, s);
}
template <int P>
__device__ __forceinline__ void store_spinor(const SpinorF& f, int i, const Spinor<typename Real<P>::T>& s)
{
    SpIO<P, true>::store(f, i, s);
}

// gauge links ----------------------------------------------------------------
template <int P>
__device__ __forceinline__ void load_link(const GaugeF& g, int mu, int par, int i, Su3<typename Real<P>::T>& u);

template <>
__device__ __forceinline__ void load_link<PREC64>(const GaugeF& g, int mu, int par, int i, Su3<double>& u)
{
    const double2* p = (const double2*)g.v + (size_t)(mu * 2 + par) * 9 * g.Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 d = __ldg(p + (size_t)k * g.Vh + i);
        u.m[k / 3][k % 3] = mk(d.x, d.y);
    }
}
template <>
__device__ __forceinline__ void load_link<PRECDF>(const GaugeF& g, int mu, int par, int i, Su3<df>& u)
{
    const double2* p = (const double2*)g.v + (size_t)(mu * 2 + par) * 9 * g.Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 d = __ldg(p + (size_t)k * g.Vh + i);
        u.m[k / 3][k % 3] = mk(df_split(d.x), df_split(d.y));
    }
}
template <>
__device__ __forceinline__ void load_link<PRECDS>(const GaugeF& g, int mu, int par, int i, Su3<df>& u)
{
    load_link<PRECDF>(g, mu, par, i, u);
}
template <>
__device__ __forceinline__ void load_link<PREC32>(const GaugeF& g, int mu, int par, int i, Su3<float>& u)
{
    const float4* p = (const float4*)g.v + (size_t)(mu * 2 + par) * 3 * g.Vh;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float4 d = __ldg(p + (size_t)k * g.Vh + i);
        u.m[(2 * k) / 3][(2 * k) % 3] = mk(d.x, d.y);
        u.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(d.z, d.w);
    }
    complete_row2(u);
}
template <>
__device__ __forceinline__ void load_link<PREC16>(const GaugeF& g, int mu, int par, int i, Su3<float>& u)
{
    const uint2* p = (const uint2*)g.v + (size_t)(mu * 2 + par) * 3 * g.Vh;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint2 d = __ldg(p + (size_t)k * g.Vh + i);
        float2 a = __half22float2(*reinterpret_cast<__half2*>(&d.x));
        float2 b = __half22float2(*reinterpret_cast<__half2*>(&d.y));
        u.m[(2 * k) / 3][(2 * k) % 3] = mk(a.x, a.y);
        u.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(b.x, b.y);
    }
    complete_row2(u);
}

// word k (elements 2k, 2k + 1 of rows 0-1) of link (mp = mu*2 + parity, i)
// in the single, half and bfloat16 copies (the bfloat16 copy follows the
// half one, 24 Vh words further)
__device__ __forceinline__ void store_low_link_word(float4* U32, uint2* U16, int Vh, int mp, int k, int i, double xr,
                                                    double xi, double yr, double yi)
{
    const size_t o = (size_t)mp * 3 * Vh + (size_t)k * Vh + i;
    U32[o] = make_float4((float)xr, (float)xi, (float)yr, (float)yi);
    __half2 hx = __floats2half2_rn((float)xr, (float)xi);
    __half2 hy = __floats2half2_rn((float)yr, (float)yi);
    U16[o] = make_uint2(*reinterpret_cast<unsigned*>(&hx), *reinterpret_cast<unsigned*>(&hy));
    __nv_bfloat162 bx = __floats2bfloat162_rn((float)xr, (float)xi);
    __nv_bfloat162 by = __floats2bfloat162_rn((float)yr, (float)yi);
    U16[(size_t)24 * Vh + o] = make_uint2(*reinterpret_cast<unsigned*>(&bx), *reinterpret_cast<unsigned*>(&by));
}

template <>
__device__ __forceinline__ void load_link<PRECBF>(const GaugeF& g, int mu, int par, int i, Su3<float>& u)
{
    const uint2* p = (const uint2*)g.v + (size_t)(mu * 2 + par) * 3 * g.Vh;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint2 d = __ldg(p + (size_t)k * g.Vh + i);
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&d.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&d.y));
        u.m[(2 * k) / 3][(2 * k) % 3] = mk(a.x, a.y);
        u.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(b.x, b.y);
    }
    complete_row2(u);
}

// ---------------------------------------------------------------------------
// the hopping term at one output site
//   mode 0: all hops (x0 wrap carries bc_t)
//   mode 1: hops inside one slab only (W1)
//   mode 2: hops between different slabs only (blocks B, C of M)
//   mode 3: hops inside one sub-slab only (W2; needs g.l0s)
//   mode 4: hops between the two sub-slabs of one slab (blocks B2, C2 of W1)
// dag = 1 gives H^dag (projectors swapped).  acc is overwritten.
// ---------------------------------------------------------------------------
enum { MODE_ALL = 0, MODE_INTRA = 1, MODE_CROSS = 2, MODE_INTRA2 = 3, MODE_CROSS2 = 4 };

// is a time-like hop across the face between slices xf-1 and xf (mod L0)
// kept in `mode`?  (space-like hops: kept unless mode is 2 or 4)
LQ_HD bool t_hop_kept(const Geo& g, int mode, int xf)
{
    if (mode == MODE_ALL) return true;
    const bool small = g.L[0] <= 64;
    const int xn = xf >= g.L[0] ? xf - g.L[0] : xf;  // xf = L0 is the face at 0
    const bool slab_face = small ? ((g.face >> xn) & 1ull) != 0 : (xf % g.l0) == 0;
    if (mode == MODE_INTRA) return !slab_face;
    if (mode == MODE_CROSS) return slab_face;
    const bool sub_face = g.l0s > 0 && (small ? ((g.sface >> xn) & 1ull) != 0 : (xf % g.l0s) == 0);
    if (mode == MODE_INTRA2) return !sub_face;
    return sub_face && !slab_face;
}

// ld(j, spinor) provides the input spinor at eo index j of parity 1-pout.
// UNR: unrolling of the loop over the four directions (4: every hop
// specialised at compile time, the fastest code for a kernel that runs one
// sweep; 1: one copy of the hop code, four times smaller, for the large
// persistent kernels whose many phases would otherwise not fit the
// instruction cache)
template <int P, int UNR = 4, class Loader>
__device__ __forceinline__ void hop_site_ld(const Geo& g, int mode, int dag, int pout, int i, Loader ld,
                                            const GaugeF& U, Spinor<typename Real<P>::T>& acc);

template <int P, bool RO, int UNR = 4>
__device__ __forceinline__ void hop_site_df(const Geo& g, int mode, int dag, int pout, int i, const SpinorF& in,
                                            const GaugeF& U, Spinor<df>& acc);

template <int P, bool RO = true, int UNR = 4>
__device__ __forceinline__ void hop_site(const Geo& g, int mode, int dag, int pout, int i,
                                         const SpinorF& in, const GaugeF& U,
                                         Spinor<typename Real<P>::T>& acc)
{
    if constexpr (P == PRECDF || P == PRECDS)
        hop_site_df<P, RO, UNR>(g, mode, dag, pout, i, in, U, acc);
    else
        hop_site_ld<P, UNR>(g, mode, dag, pout, i,
                            [&](int j, Spinor<typename Real<P>::T>& s) { load_spinor<P, RO>(in, j, s); }, U, acc);
}

template <int P, int UNR, class Loader>
__device__ __forceinline__ void hop_site_ld(const Geo& g, int mode, int dag, int pout, int i, Loader ld,
                                            const GaugeF& U, Spinor<typename Real<P>::T>& acc)
{
    typedef typename Real<P>::T T;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc.c[s][c] = mk(T(0), T(0));
    int x[4];
    eo_coords(g, pout, i, x);
    const int lex = lex_of(g, x);
    int stride = 1;
    const int pin = 1 - pout;
#pragma unroll(UNR)
    for (int mu = 3; mu >= 0; --mu) {
        // forward hop x -> x + mu
        {
            int nl = lex + stride;
            bool wrap = (x[mu] == g.L[mu] - 1);
            if (wrap) nl -= g.L[mu] * stride;
            bool use = true;
            if (mu == 0) use = t_hop_kept(g, mode, x[0] + 1);
            else if (mode == MODE_CROSS || mode == MODE_CROSS2) use = false;
            if (use) {
                Spinor<T> ps;
                ld(nl >> 1, ps);
                Su3<T> u;
                load_link<P>(U, mu, pout, i, u);
                HalfSp<T> h, w;
                const int sg = dag ? +1 : -1;
                project(mu, sg, ps, h);
                su3_mul_half(u, h, w);
                if (mu == 0 && wrap && g.bc_t < 0) {
#pragma unroll
                    for (int s = 0; s < 2; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) w.c[s][c] = -w.c[s][c];
                }
                accum_recon(mu, sg, w, acc);
            }
        }
        // backward hop x -> x - mu
        {
            int nl = lex - stride;
            bool wrap = (x[mu] == 0);
            if (wrap) nl += g.L[mu] * stride;
            bool use = true;
            if (mu == 0) use = t_hop_kept(g, mode, x[0]);
            else if (mode == MODE_CROSS || mode == MODE_CROSS2) use = false;
            if (use) {
                Spinor<T> ps;
                ld(nl >> 1, ps);
                Su3<T> u;
                load_link<P>(U, mu, pin, nl >> 1, u);
                HalfSp<T> h, w;
                const int sg = dag ? -1 : +1;
                project(mu, sg, ps, h);
                su3_dagmul_half(u, h, w);
                if (mu == 0 && wrap && g.bc_t < 0) {
#pragma unroll
                    for (int s = 0; s < 2; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) w.c[s][c] = -w.c[s][c];
                }
                accum_recon(mu, sg, w, acc);
            }
        }
        stride *= g.L[mu];
    }
}

// The hopping term in double-float arithmetic, arranged for registers: a
// neighbour is projected colour by colour as its components arrive (the
// full spinor is never held), and the link is applied row by row (column
// by column for U^dag), each row's result accumulated at once.  Same
// operations as hop_site_ld, about 90 instead of 130 live registers.
template <int P, bool RO>
__device__ __forceinline__ cx<df> df_in(const SpinorF& f, int c, int j)
{
    if constexpr (P == PRECDS) {
        const float4 d = ldv<float4, RO>((const float4*)f.v + (size_t)c * f.N + j);
        return mk(df(d.x, d.z), df(d.y, d.w));
    } else {
        const double2 d = ldv<double2, RO>((const double2*)f.v + (size_t)c * f.N + j);
        return mk(df_split(d.x), df_split(d.y));
    }
}

__device__ __forceinline__ cx<df> df_link(const double2* p, int k, int Vh, int i)
{
    const double2 d = __ldg(p + (size_t)k * Vh + i);
    return mk(df_split(d.x), df_split(d.y));
}

template <int P, bool RO, int UNR>
__device__ __forceinline__ void hop_site_df(const Geo& g, int mode, int dag, int pout, int i, const SpinorF& in,
                                            const GaugeF& U, Spinor<df>& acc)
{
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc.c[s][c] = mk(df(0), df(0));
    int x[4];
    eo_coords(g, pout, i, x);
    const int lex = lex_of(g, x);
    int stride = 1;
    const int pin = 1 - pout;
#pragma unroll(UNR)
    for (int mu = 3; mu >= 0; --mu) {
#pragma unroll
        for (int fw = 1; fw >= 0; --fw) {
            int nl = fw ? lex + stride : lex - stride;
            const bool wrap = fw ? (x[mu] == g.L[mu] - 1) : (x[mu] == 0);
            if (wrap) nl += fw ? -g.L[mu] * stride : g.L[mu] * stride;
            bool use = true;
            if (mu == 0) use = t_hop_kept(g, mode, fw ? x[0] + 1 : x[0]);
            else if (mode == MODE_CROSS || mode == MODE_CROSS2) use = false;
            if (!use) continue;
            const int j = nl >> 1;
            const int sg = fw ? (dag ? +1 : -1) : (dag ? -1 : +1);
            HalfSp<df> h;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                project1(mu, sg, df_in<P, RO>(in, c, j), df_in<P, RO>(in, 3 + c, j), df_in<P, RO>(in, 6 + c, j),
                         df_in<P, RO>(in, 9 + c, j), h.c[0][c], h.c[1][c]);
            // forward: U_mu(x) at this site; backward: U_mu(x - mu)^dag
            const double2* up = (const double2*)U.v + (size_t)(mu * 2 + (fw ? pout : pin)) * 9 * U.Vh;
            const int li = fw ? i : j;
            const bool neg = mu == 0 && wrap && g.bc_t < 0;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cx<df> w0, w1;
                if (fw) {
                    const cx<df> u0 = df_link(up, 3 * r, U.Vh, li), u1 = df_link(up, 3 * r + 1, U.Vh, li),
                                 u2 = df_link(up, 3 * r + 2, U.Vh, li);
                    w0 = u0 * h.c[0][0] + u1 * h.c[0][1] + u2 * h.c[0][2];
                    w1 = u0 * h.c[1][0] + u1 * h.c[1][1] + u2 * h.c[1][2];
                } else {
                    const cx<df> u0 = df_link(up, r, U.Vh, li), u1 = df_link(up, 3 + r, U.Vh, li),
                                 u2 = df_link(up, 6 + r, U.Vh, li);
                    w0 = cjmul(u0, h.c[0][0]) + cjmul(u1, h.c[0][1]) + cjmul(u2, h.c[0][2]);
                    w1 = cjmul(u0, h.c[1][0]) + cjmul(u1, h.c[1][1]) + cjmul(u2, h.c[1][2]);
                }
                if (neg) {
                    w0 = -w0;
                    w1 = -w1;
                }
                accum_recon1(mu, sg, w0, w1, acc, r);
            }
        }
        stride *= g.L[mu];
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Profiler {
    unsigned on = 0;  // bit mask of the kernel ids being timed
    struct Rec {
        cudaEvent_t a, b;
        int id;
        double bytes;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    int64_t launches[5] = {0, 0, 0, 0, 0};
    double ms[5] = {0, 0, 0, 0, 0};
    double bytes[5] = {0, 0, 0, 0, 0};
    std::vector<float> hist[5];  // per-launch device times since the last reset
    std::vector<Rec> graph_recs;  // event pairs recorded inside the MD graph
};

struct Work;  // solver workspace (lqcd_solver.cu)

// launch schedules picked by lqcd_autotune (defaults until it runs)
struct Tune {
    int hop_bs[NPREC] = {128, 128, 128, 128};  // k_hop threads per block, per precision
    int solve_spt[NPREC][2] = {{1, 1}, {1, 1}, {1, 1}, {1, 1}};  // k_solve sites per thread [prec][block, global]
    int cluster_series = 0;  // single-precision slab series on thread-block clusters (opt-in: slower on GB300)
};

struct lqcd_ctx {
    Geo g;   // active geometry (level 1, or level 2 inside a GeoScope)
    Geo g1;  // level 1: slabs of thickness l0 (g1.l0s: sub-slabs, or 0)
    cudaStream_t stream;
    int device;
    int num_sms;
    std::string err;
    bool have_gauge = false;
    // internal gauge copies
    double2* U64 = nullptr;  // [4][2][9][Vh]
    float4* U32 = nullptr;   // [4][2][3][Vh]
    uint2* U16 = nullptr;    // [4][2][3][Vh] fp16, then [4][2][3][Vh] bf16
    double2* U64_save = nullptr;
    // double full-lattice spinor scratch fields [2][12][Vh]
    std::vector<double2*> f64;
    // momenta / force scratch [4][V][8]
    double* P = nullptr;
    double* F = nullptr;
    // boundary scratch
    double* bnd[4] = {nullptr, nullptr, nullptr, nullptr};
    // reductions
    double* red_part = nullptr;  // partial sums
    double* red_out = nullptr;   // device scalars
    double* red_host = nullptr;  // pinned host mirror
    int red_blocks = 0;
    Work* work = nullptr;
    Profiler prof;
    Tune tune;
    double* d_sscale = nullptr;  // step-size table [2][L0] of the current MD
    int64_t launches = 0;    // kernels launched by this handle
    bool deferred = false;   // solves leave status on the device (graph capture)
    bool capturing = false;  // a CUDA graph is being recorded: no profiling
    // the molecular dynamics of one trajectory as a CUDA graph
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t md_exec = nullptr;
    std::vector<unsigned char> md_key;  // parameters the graph was recorded for
    int64_t md_launches = 0;            // kernels per replay
    // chronological initial guesses of the MD's solves: per solve site of
    // the force terms the even halves of its last chrono_depth solutions
    // (buffers CHRONO_MAX k + j, a ring; chrono_cur[k] names the newest)
    // and the MD times of the links each buffer's solution was solved on
    static constexpr int NCHRONO = 12;
    static constexpr int NMRE = 6;        // solutions of a minimal-residual guess
    static constexpr int CHRONO_MAX = NMRE;
    double2* chrono_buf[CHRONO_MAX * NCHRONO] = {};
    int chrono_n[NCHRONO] = {};    // solutions kept (0 .. chrono_depth[k])
    int chrono_cur[NCHRONO] = {};
    double chrono_t[NCHRONO][CHRONO_MAX] = {};  // MD time of each buffer
    int chrono_depth[NCHRONO] = {};  // solutions kept per slot: chrono + 1 (at most 3), NMRE for
                                     // the minimal-residual slots of the whole-lattice solves
    bool chrono_mre = false;         // chrono = 3: whole-lattice solves guess by minimal residual
    // workspace of the minimal-residual guess (lqcd_chrono.cu)
    float4* mre_w[NMRE] = {};
    float4* mre_v = nullptr;
    float4* mre_o = nullptr;
    double2* mre_c = nullptr;
    double* mre_part = nullptr;
    double md_time = 0.0;              // MD time of the links in do_md
    bool chrono_frozen = false;        // guesses are read but not replaced
    int md_nforce = 0;                  // force evaluations per replay
    int md_solves = 0;                  // solves per replay
    int64_t iter_count = 0;  // inner iterations since reset (trajectory stats)
    int64_t site_iters = 0;  // inner iterations x even sites of the system
    int64_t hop_sites = 0;   // half-lattice hopping site updates of those iterations
    int solve_count = 0;
    // clock64 cycles a CTA of the persistent solver waits at a barrier
    // before the solve gives up with LQCD_ERR_TIMEOUT (lqcd_set_wait_limit)
    static constexpr long long WAIT_LIMIT_DEFAULT = 4000000000LL;  // ~2 s
    long long wait_limit = WAIT_LIMIT_DEFAULT;
    // inner iteration of every whole-lattice solve (M^-1 of the boundary
    // term, lqcd_solve_wilson): SOLVER_BICGSTAB or SOLVER_SAP with sap_terms
    // series terms per slab solve (lqcd_set_global_solver)
    int global_method = 0;
    int sap_terms = 4;
};

// switches the handle to another geometry for the lifetime of the scope
struct GeoScope {
    lqcd_ctx* h;
    Geo saved;
    GeoScope(lqcd_ctx* hh, const Geo& g) : h(hh), saved(hh->g) { h->g = g; }
    ~GeoScope() { h->g = saved; }
};

// error helpers
#define LQ_CUDA(h, call)                                                                    \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return LQCD_ERR_CUDA;                                                           \
        }                                                                                   \
    } while (0)

#define LQ_TRY(x)                 \
    do {                          \
        int st_ = (x);            \
        if (st_ != LQCD_OK) return st_; \
    } while (0)

// profiling hooks
void prof_begin(lqcd_ctx* h, int id, cudaEvent_t* a);
void prof_end(lqcd_ctx* h, int id, cudaEvent_t a, double bytes);

// ---------------------------------------------------------------------------
// internal host API shared by the translation units
// ---------------------------------------------------------------------------
SpinorF sp_view(const void* base, int prec, int parity, int Vh, float* nrm_base);
inline SpinorF sp64(double2* base, int parity, int Vh)
{
    SpinorF f;
    f.v = base + (size_t)parity * 12 * Vh;
    f.nrm = nullptr;
    f.N = Vh;
    return f;
}
GaugeF gauge_view(lqcd_ctx* h, int prec);

// fields.cu
int pack_spinor(lqcd_ctx* h, double2* dst, const double* abi, int parity_first, int nparity);
int unpack_spinor(lqcd_ctx* h, double* abi, const double2* src, int parity_first, int nparity);
int pack_gauge(lqcd_ctx* h, const double* abi);
int unpack_gauge(lqcd_ctx* h, double* abi);
int convert_spinor(lqcd_ctx* h, SpinorF dst, int dprec, SpinorF src, int sprec, int n);
int index_maps(lqcd_ctx* h, int32_t* maps);
// boundary space of the active geometry; nface = 2: both faces of every
// black slab (level 1), nface = 1: first slice only (level 2)
int embed_boundary(lqcd_ctx* h, double2* full, const double* coords, int nface = 2);
int project_boundary(lqcd_ctx* h, double* coords, const double2* full, int nface = 2);
int axpby_full(lqcd_ctx* h, double2* y, double a, const double2* x, double b, int colour);
int gamma5_full(lqcd_ctx* h, double2* y, const double2* x);
// even half: y = gamma5^g5 (a x1 + b x0); x0 not read when b = 0
int lincomb_even(lqcd_ctx* h, double2* y, double a, const double2* x1, double b, const double2* x0, int g5);
// chrono.cu: minimal-residual guess x_e for (1 - kappa^2 H_eo H_oe) x_e = b_e
// from the n solutions sol[i] (double even halves, gamma5^dag applied to
// them), its workspace
int chrono_mre_guess(lqcd_ctx* h, const double2* const* sol, int n, double2* x_e, const double2* b_e, double kappa,
                     int dag);
int chrono_mre_alloc(lqcd_ctx* h);
void chrono_mre_free(lqcd_ctx* h);
// even half: y = gamma5^g5 (a x2 + b x1 + c x0)
int lincomb3_even(lqcd_ctx* h, double2* y, double a, const double2* x2, double b, const double2* x1, double c,
                  const double2* x0, int g5);
int keep_colour(lqcd_ctx* h, double2* y, int colour);
int norm2_dev(lqcd_ctx* h, const double* x, int64_t n, double* dev_out);
int rng_normals(lqcd_ctx* h, double* out, int64_t n, uint64_t seed, uint32_t stream, uint32_t traj,
                double scale);
int rng_spinor(lqcd_ctx* h, double2* full, uint64_t seed, uint32_t stream, uint32_t traj);
int read_scalars(lqcd_ctx* h, int n, double* host);

// dslash.cu
// out(p_out) = a * x(p_out) + c * H_{p_out,1-p_out} in(1-p_out) on the output
// sites of slabs with the given colour (-1: all); x may be null (a ignored)
int hop_sweep(lqcd_ctx* h, int prec, int mode, int dag, int pout, int colour, SpinorF out,
              SpinorF in, double a, SpinorF x, double c);

// solver.cu
int solver_init(lqcd_ctx* h);
// the Schwarz-preconditioned solve's workspace (11 full-lattice vectors),
// allocated once, outside any graph capture
int solver_sap_alloc(lqcd_ctx* h);
void solver_free(lqcd_ctx* h);
// sticky status and iteration sums of the solves since the last call
// (site_iters: BiCGstab iterations x system sites; series_sites: the same
// for geometric-series iterations)
int solver_collect(lqcd_ctx* h, int64_t* iters, int64_t* site_iters, int64_t* outer_sites = nullptr,
                   int64_t* series_sites = nullptr, int64_t* sap_sites = nullptr);
// algorithmic bytes per system site of one inner iteration / outer cycle
// (nsap: series terms of the Schwarz preconditioner, SOLVER_SAP only)
void solver_site_bytes(int prec, int method, double* inner, double* outer, int nsap = 0);
// even-odd reduced solve (1 - kappa^2 H_eo H_oe) x_e = b_e on the slabs of
// `colour` (block mode) or globally; x_e, b_e: double parity-0 views
// `diag` replaces the 1 of the system: diag - kappa^2 H_eo H_oe (W3,eo = W2,eo + rho)
// `method`: inner iteration, BiCGstab or the geometric series (which needs
// the spectral radius of kappa^2 H_eo H_oe / diag below one)
// SOLVER_SAP (whole-lattice solves only): BiCGstab on M preconditioned by
// one multiplicative Schwarz cycle over the red / black x0-slabs;
// SOLVER_SAPB: the same over red / black 4-D blocks of at most 4^4 sites,
// each block solved by one CTA in shared memory
enum { SOLVER_BICGSTAB = 0, SOLVER_SERIES = 1, SOLVER_SAP = 2, SOLVER_SAPB = 3 };
// half-lattice hopping site updates per inner iteration and even site of
// the system: BiCGstab 4, series 2, Schwarz-preconditioned BiCGstab two
// applications of (red and black slab solves of nsap series terms, 2 + 2
// nsap half sweeps, and M, 2 half sweeps)
inline int solver_hops_per_iter(int method, int nsap)
{
    return method == SOLVER_SERIES ? 2 : (method == SOLVER_SAP || method == SOLVER_SAPB) ? 4 * (2 + nsap) : 4;
}
// `guess`: 1 if x_e holds an initial guess (its residual is computed in
// double before the first inner cycle), 0 to start from x = 0
int eo_solve(lqcd_ctx* h, int mode, int colour, int prec, double kappa, double2* x_e,
             const double2* b_e, double tol, int max_iter, int* iters_sys, double* resid_sys,
             double diag = 1.0, int method = SOLVER_BICGSTAB, int guess = 0);

// force.cu
// prec: PREC64 runs the link arithmetic in double, otherwise in single
// precision on the single-precision links (results accumulated in double).
// ss: device step-size table [2][L0] (row 0 space-like, row 1 time-like
// links) multiplying each link's contribution, or null for s = 1.
int force_bilinear(lqcd_ctx* h, double* F, const double2* a1, const double2* b1, int mask1,
                   double coef1, const double2* a2, const double2* b2, int mask2, double coef2, int prec,
                   const double* ss = nullptr);
int gauge_force_kick(lqcd_ctx* h, double* F, double coef, int prec, const double* ss = nullptr);
int plaquette_sum(lqcd_ctx* h, double* dev_out);
int force_profile(lqcd_ctx* h, const double* F, double* out);
int update_links(lqcd_ctx* h, const double* P, double dt, const double* ss = nullptr);
int roll_links(lqcd_ctx* h, int shift);
int kinetic_sum(lqcd_ctx* h, const double* P, double* dev_out);
int refresh_low_precision(lqcd_ctx* h);
