// lqcd_dslash.cu -- the hopping term of eq. (2) as one sweep over the output
// sites of one parity: out = a x + c H_{p,1-p} in, optionally restricted to
// the hops inside one x0-slab (W1) or between slabs (the blocks B, C of M),
// and to the output sites of the slabs of one colour.
//
// One thread per output site.  Every neighbour is read as a full spinor
// with 128-bit (single: float4, half: uint4) or 2x64-bit (double2) loads of
// consecutive sites, spin-projected to a half spinor, multiplied by the
// (rebuilt) link and accumulated; the output is written once.
#include <algorithm>

#include "lqcd_common.cuh"

namespace {

// block size chosen at run time (lqcd_autotune), at most HOP_BS_MAX
constexpr int HOP_BS_MAX = 256;

// acc += sc (1 + sg gamma_mu) psi rebuilt from its upper half w (the
// multiplication by sc fused into the accumulation)
__device__ __forceinline__ void accum_recon_sc(int mu, int sg, const HalfSp<float>& w, float sc, Spinor<float>& acc)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        cx<float> l0, l1;
        switch (mu) {
            case 0: l0 = -w.c[0][i]; l1 = -w.c[1][i]; break;
            case 1: l0 = mul_i(w.c[1][i]); l1 = mul_i(w.c[0][i]); break;
            case 2: l0 = w.c[1][i]; l1 = -w.c[0][i]; break;
            default: l0 = mul_i(w.c[0][i]); l1 = mul_mi(w.c[1][i]); break;
        }
        const float sl = sg < 0 ? -sc : sc;
        acc.c[0][i] = mk(acc.c[0][i].re + sc * w.c[0][i].re, acc.c[0][i].im + sc * w.c[0][i].im);
        acc.c[1][i] = mk(acc.c[1][i].re + sc * w.c[1][i].re, acc.c[1][i].im + sc * w.c[1][i].im);
        acc.c[2][i] = mk(acc.c[2][i].re + sl * l0.re, acc.c[2][i].im + sl * l0.im);
        acc.c[3][i] = mk(acc.c[3][i].re + sl * l1.re, acc.c[3][i].im + sl * l1.im);
    }
}

// the hopping term at one output site for half storage: each neighbour is
// converted without its per-site scale, projected and multiplied by the
// link, and the scale (with the x0 boundary sign) enters once, in the
// accumulation: the same sum as hop_site<PREC16> with 24 fewer
// multiplications per hop
__device__ __forceinline__ void hop_site_h16(const Geo& g, int mode, int dag, int pout, int i, const SpinorF& in,
                                             const GaugeF& U, Spinor<float>& acc)
{
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc.c[s][c] = mk(0.f, 0.f);
    int x[4];
    eo_coords(g, pout, i, x);
    const int lex = lex_of(g, x);
    int stride = 1;
    const int pin = 1 - pout;
    const uint4* pv = (const uint4*)in.v;
    auto ld = [&](int j, Spinor<float>& sp) -> float {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 d = __ldg(pv + (size_t)k * in.N + j);
            const unsigned w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w[q]));
                const int cc = 4 * k + q;
                sp.c[cc / 3][cc % 3] = mk(v.x, v.y);
            }
        }
        return __ldg(in.nrm + j);
    };
#pragma unroll
    for (int mu = 3; mu >= 0; --mu) {
        {
            int nl = lex + stride;
            const bool wrap = (x[mu] == g.L[mu] - 1);
            if (wrap) nl -= g.L[mu] * stride;
            bool use = true;
            if (mu == 0) use = t_hop_kept(g, mode, x[0] + 1);
            else if (mode == MODE_CROSS || mode == MODE_CROSS2) use = false;
            if (use) {
                Spinor<float> ps;
                float sc = ld(nl >> 1, ps);
                Su3<float> u;
                load_link<PREC16>(U, mu, pout, i, u);
                HalfSp<float> h, w;
                const int sg = dag ? +1 : -1;
                project(mu, sg, ps, h);
                su3_mul_half(u, h, w);
                if (mu == 0 && wrap && g.bc_t < 0) sc = -sc;
                accum_recon_sc(mu, sg, w, sc, acc);
            }
        }
        {
            int nl = lex - stride;
            const bool wrap = (x[mu] == 0);
            if (wrap) nl += g.L[mu] * stride;
            bool use = true;
            if (mu == 0) use = t_hop_kept(g, mode, x[0]);
            else if (mode == MODE_CROSS || mode == MODE_CROSS2) use = false;
            if (use) {
                Spinor<float> ps;
                float sc = ld(nl >> 1, ps);
                Su3<float> u;
                load_link<PREC16>(U, mu, pin, nl >> 1, u);
                HalfSp<float> h, w;
                const int sg = dag ? -1 : +1;
                project(mu, sg, ps, h);
                su3_dagmul_half(u, h, w);
                if (mu == 0 && wrap && g.bc_t < 0) sc = -sc;
                accum_recon_sc(mu, sg, w, sc, acc);
            }
        }
        stride *= g.L[mu];
    }
}

template <int P>
__device__ __forceinline__ void hop_body(Geo g, int mode, int dag, int pout, int colour, SpinorF out, SpinorF in,
                                         GaugeF U, double a, SpinorF x, double c, int nsites)
{
    typedef typename Real<P>::T T;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nsites) return;
    int i = t;
    if (colour >= 0) {
        const int k = t / g.Sh;
        i = (colour + 2 * k) * g.Sh + (t - k * g.Sh);
    }
    Spinor<T> acc;
    if constexpr (P == PREC16)
        hop_site_h16(g, mode, dag, pout, i, in, U, acc);
    else
        hop_site<P>(g, mode, dag, pout, i, in, U, acc);
    const T cc = (T)c;
    if (x.v) {
        Spinor<T> xs;
        load_spinor<P>(x, i, xs);
        const T aa = (T)a;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc.c[s][q] = aa * xs.c[s][q] + cc * acc.c[s][q];
    } else {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc.c[s][q] = cc * acc.c[s][q];
    }
    store_spinor<P>(out, i, acc);
}

template <int P>
__global__ void __launch_bounds__(HOP_BS_MAX) k_hop(Geo g, int mode, int dag, int pout, int colour, SpinorF out,
                                               SpinorF in, GaugeF U, double a, SpinorF x, double c, int nsites)
{
    hop_body<P>(g, mode, dag, pout, colour, out, in, U, a, x, c, nsites);
}

// the double-float sweep: its long dependent chains want more resident
// warps than its natural register count allows
__global__ void __launch_bounds__(HOP_BS_MAX, 2) k_hop_df(Geo g, int mode, int dag, int pout, int colour, SpinorF out,
                                                     SpinorF in, GaugeF U, double a, SpinorF x, double c, int nsites)
{
    hop_body<PRECDF>(g, mode, dag, pout, colour, out, in, U, a, x, c, nsites);
}

}  // namespace

// algorithmic DRAM bytes of one output site: the output, the input site and
// the eight links, each moved once (neighbour spinors reused from cache)
double hop_site_bytes(int prec, bool with_x)
{
    const bool dbl = prec == PREC64 || prec == PRECDF;
    const double sp = dbl ? 192.0 : prec == PREC32 ? 96.0 : prec == PREC16 ? 52.0 : 48.0;
    const double lk = dbl ? 144.0 : prec == PREC32 ? 48.0 : 24.0;
    return 2.0 * sp + 8.0 * lk + (with_x ? sp : 0.0);
}

int hop_sweep(lqcd_ctx* h, int prec, int mode, int dag, int pout, int colour, SpinorF out, SpinorF in,
              double a, SpinorF x, double c)
{
    const Geo& g = h->g;
    const int nsites = colour < 0 ? g.Vh : (g.nb / 2) * g.Sh;
    const int bs = std::min(std::max(h->tune.hop_bs[prec == PRECDF ? PREC64 : prec], 32), HOP_BS_MAX);
    const int nb = (nsites + bs - 1) / bs;
    GaugeF U = gauge_view(h, prec);
    cudaEvent_t ev;
    prof_begin(h, 0, &ev);
    if (prec == PREC64)
        k_hop<PREC64><<<nb, bs, 0, h->stream>>>(g, mode, dag, pout, colour, out, in, U, a, x, c, nsites);
    else if (prec == PRECDF)
        k_hop_df<<<nb, bs, 0, h->stream>>>(g, mode, dag, pout, colour, out, in, U, a, x, c, nsites);
    else if (prec == PREC32)
        k_hop<PREC32><<<nb, bs, 0, h->stream>>>(g, mode, dag, pout, colour, out, in, U, a, x, c, nsites);
    else if (prec == PREC16)
        k_hop<PREC16><<<nb, bs, 0, h->stream>>>(g, mode, dag, pout, colour, out, in, U, a, x, c, nsites);
    else
        k_hop<PRECBF><<<nb, bs, 0, h->stream>>>(g, mode, dag, pout, colour, out, in, U, a, x, c, nsites);
    h->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->err = std::string("hop kernel: ") + cudaGetErrorString(e);
        return LQCD_ERR_CUDA;
    }
    prof_end(h, 0, ev, hop_site_bytes(prec, x.v != nullptr) * nsites);
    return LQCD_OK;
}
