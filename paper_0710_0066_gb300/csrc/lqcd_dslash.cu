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
