// domain.cu -- the Dslash on one time slab of a domain-decomposed lattice (Sec. 4: every
// sub-lattice holds its bulk plus a halo of the neighbours' boundary sites, exchanged once
// per operator application).
//
// The global lattice Nx x Ny x Nz x Nt is cut into slabs of lt time slices, [t0, t0 + lt),
// t0 and lt even (so a site's parity in the slab's own even-odd order equals its global
// parity).  The HISQ stencil reaches three slices across a cut (the Naik hop), so the
// Dslash of a slab needs the input field of the opposite parity on the three slices below
// t0 and the three slices from t0 + lt up: the halos.  With t slowest in the even-odd
// order, one parity of one time slice is a contiguous run of F = Nx Ny Nz / 2 half-sites
// (half index h + F t for the face index h = (x + Nx (y + Ny z)) / 2), so the three slices
// a neighbour needs are one contiguous block: "packing" a halo is a copy of 3F records, and
// the received blocks are read in place by the slab's Dslash kernel.
//
// Links never change: at creation the slab takes, from the global link field, its own links
// (all four directions) and the time-direction links of the three slices below it (their
// backward hops end inside the slab).  Staggered phases and the antiperiodic time boundary
// are folded in by GLOBAL position: a k-hop link U_t(T) carries the boundary sign when
// T + k >= Nt, as in an undivided lattice.  The slab's own links live in an ordinary
// context's link store (phased input), the halo links in a small array.
#include <cstring>
#include <string>

#include "arith.cuh"
#include "dslash.cuh"

namespace hisq {

struct DdGeom {
    int g[4];      // global dims
    int t0, lt;    // slab
    uint32_t F;    // sites of one parity in one time slice
    uint32_t Vs;   // sites of one time slice (both parities)
};

// global canonical index (Sec. 4.3 even-odd order) of (x, y, z, t)
__device__ __forceinline__ size_t dd_global_index(const DdGeom &d, int x, int y, int z, int t)
{
    const size_t lex = (size_t)x + (size_t)d.g[0] * ((size_t)y + (size_t)d.g[1] * ((size_t)z + (size_t)d.g[2] * t));
    const size_t V = (size_t)d.g[0] * d.g[1] * d.g[2] * d.g[3];
    return lex / 2 + ((x + y + z + t) & 1) * (V / 2);
}

// sign of link type (0 fat, 1 long) in direction mu at global (x, y, z, t): MILC eta_mu and
// the antiperiodic time boundary on the hop that crosses t = Nt
__device__ __forceinline__ double dd_sign(const DdGeom &d, int x, int y, int z, int t, int mu, int type)
{
    int neg = 0;
    if (mu == 1) neg = x & 1;
    else if (mu == 2) neg = (x + y) & 1;
    else if (mu == 3) neg = ((x + y + z) & 1) ^ (t + (type ? 3 : 1) >= d.g[3]);
    return neg ? -1.0 : 1.0;
}

// the slab's links in its own canonical order [4][Vloc][18], phased by global position
__global__ void k_dd_slab_links(const DdGeom d, const double *gfat, const double *glng, double *lfat, double *llng)
{
    const size_t Vloc = (size_t)d.Vs * d.lt;
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (i >= Vloc) return;
    // local canonical index i -> local (x, y, z, tl): parity block, then half index
    const size_t Vh = Vloc / 2;
    const int p = i >= Vh;
    const size_t s = i - p * Vh;
    const int nxh = d.g[0] / 2;
    const int xh = (int)(s % nxh);
    size_t r = s / nxh;
    const int y = (int)(r % d.g[1]);
    r /= d.g[1];
    const int z = (int)(r % d.g[2]);
    const int tl = (int)(r / d.g[2]);
    const int t = d.t0 + tl;
    const int x = 2 * xh + ((p + y + z + tl) & 1);
    const size_t V = (size_t)d.g[0] * d.g[1] * d.g[2] * d.g[3];
    const size_t gi = dd_global_index(d, x, y, z, t);
    for (int type = 0; type < 2; type++) {
        const double sg = dd_sign(d, x, y, z, t, mu, type);
        const double *src = (type ? glng : gfat) + ((size_t)mu * V + gi) * 18;
        double *dst = (type ? llng : lfat) + ((size_t)mu * Vloc + i) * 18;
        for (int k = 0; k < 18; k++) dst[k] = sg * src[k];
    }
}

// time-direction links of the global slices T = t0 - 3 .. t0 - 1 (mod Nt):
// halo[type][j][x + Nx (y + Ny z)][18]
__global__ void k_dd_halo_links(const DdGeom d, const double *gfat, const double *glng, double *halo)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (q >= d.Vs) return;
    const int x = (int)(q % d.g[0]);
    const int y = (int)((q / d.g[0]) % d.g[1]);
    const int z = (int)(q / ((uint32_t)d.g[0] * d.g[1]));
    const int t = ((d.t0 - 3 + j) % d.g[3] + d.g[3]) % d.g[3];
    const size_t V = (size_t)d.g[0] * d.g[1] * d.g[2] * d.g[3];
    const size_t gi = dd_global_index(d, x, y, z, t);
    for (int type = 0; type < 2; type++) {
        const double sg = dd_sign(d, x, y, z, t, 3, type);
        const double *src = (type ? glng : gfat) + ((size_t)3 * V + gi) * 18;
        double *dst = halo + (((size_t)type * 3 + j) * d.Vs + q) * 18;
        for (int k = 0; k < 18; k++) dst[k] = sg * src[k];
    }
}

struct DdArgs {
    Geom g;                  // the slab's geometry (local dims Nx, Ny, Nz, lt)
    int p;                   // output parity
    const char *links;       // the slab's FP64 link store (18 reals, phases folded in)
    size_t slot_bytes;
    const double *halo_links; // [2][3][Vs][18]
    const char *in;          // slab field of parity 1 - p, canonical [Vh] records of 48 bytes
    const char *lo, *hi;     // received halos of parity 1 - p: [3][F] records, slices t0-3..t0-1
                             // and t0+lt..t0+lt+2
    char *out;               // slab field of parity p
    uint32_t F, Vs;
};

// out(x) = sum_mu [ X_mu(x) phi(x+mu) - X_mu(x-mu)^+ phi(x-mu) + W_mu(x) phi(x+3mu)
//                   - W_mu(x-3mu)^+ phi(x-3mu) ]  for every site x of parity p in the slab;
// time neighbours outside the slab come from the halos, the links of backward time hops
// that start below the slab from the halo links.  One thread per output site, FP64.
__global__ void __launch_bounds__(128) k_dd_dslash(const DdArgs a)
{
    using T = Prec<HISQ_F64>;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.g.Vh) return;
    const Site c = site_coords(a.g, s, a.p);
    const uint32_t h = s - a.F * (uint32_t)c.t;                      // face index of (x, y, z)
    const uint32_t q = (uint32_t)c.x + (uint32_t)a.g.n[0] * ((uint32_t)c.y + (uint32_t)a.g.n[1] * (uint32_t)c.z);
    const int lt = a.g.n[3];
    typename T::Acc acc;
    T::zero(acc);
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
#pragma unroll
        for (int hop = 0; hop < 4; hop++) {
            const int k = hop == 0 ? 1 : hop == 1 ? -1 : hop == 2 ? 3 : -3;
            const int type = hop >> 1;
            const bool back = hop & 1;
            const char *src = a.in;
            uint32_t sn;
            bool halo_link = false;
            if (mu < 3) {
                bool wrap;
                sn = neighbour(a.g, c, s, mu, k, wrap);
            } else {
                const int tn = c.t + k;
                if (tn < 0) {
                    src = a.lo;
                    sn = (uint32_t)(tn + 3) * a.F + h;
                    halo_link = back; // its link belongs to a slice below the slab
                } else if (tn >= lt) {
                    src = a.hi;
                    sn = (uint32_t)(tn - lt) * a.F + h;
                } else {
                    sn = (uint32_t)((int)s + k * (int)a.F);
                }
            }
            typename T::Link U;
            if (halo_link) {
                const double *L = a.halo_links + (((size_t)type * 3 + (size_t)(c.t + k + 3)) * a.Vs + q) * 18;
#pragma unroll
                for (int i = 0; i < 18; i++) U.v[i] = __ldg(L + i);
            } else {
                const int lp = back ? 1 - a.p : a.p;
                const char *slot = a.links + (size_t)((lp * 2 + type) * 4 + mu) * a.slot_bytes;
                uint32_t w[36];
                load_link_words<144>(slot, back ? sn : s, w);
                T::template unpack<18>(w, U);
            }
            typename T::Vec v;
            T::load(src, sn, v);
            if (back) T::template hop<true, true>(acc, U, v);
            else T::template hop<false, false>(acc, U, v);
        }
    }
    T::store(a.out, s, acc);
}

}  // namespace hisq

using namespace hisq;

struct hisq_dd {
    hisq_ctx *slab = nullptr;
    DdGeom d{};
    double *halo_links = nullptr;
    int device = 0;
    std::string msg;
};

static int dd_fail(hisq_dd *dd, int code, const std::string &m)
{
    if (dd) dd->msg = m;
    return code;
}

extern "C" {

void hisq_dd_destroy(hisq_dd *dd)
{
    if (!dd) return;
    cudaSetDevice(dd->device);
    cudaDeviceSynchronize();
    if (dd->halo_links) cudaFree(dd->halo_links);
    if (dd->slab) hisq_destroy(dd->slab);
    delete dd;
}

const char *hisq_dd_last_error_message(const hisq_dd *dd) { return dd ? dd->msg.c_str() : "null domain"; }
long hisq_dd_half_volume(const hisq_dd *dd) { return dd ? (long)dd->d.Vs * dd->d.lt / 2 : 0; }
long hisq_dd_halo_sites(const hisq_dd *dd) { return dd ? 3L * dd->d.F : 0; }

int hisq_dd_create(hisq_dd **out, const int gdims[4], int t0, int lt, const double *fat, const double *lng,
                   const hisq_opts *opts_in)
{
    if (!out) return HISQ_EINVAL;
    *out = nullptr;
    if (!gdims || !fat || !lng) return HISQ_EINVAL;
    hisq_opts opts;
    if (opts_in) opts = *opts_in;
    else hisq_opts_default(&opts);
    for (int i = 0; i < 4; i++)
        if (gdims[i] < 4 || (gdims[i] & 1)) return HISQ_EINVAL;
    if (opts.links_phased || lt < 4 || (lt & 1) || t0 < 0 || (t0 & 1) || t0 + lt > gdims[3]) return HISQ_EINVAL;
    hisq_dd *dd = new hisq_dd();
    dd->device = opts.device;
    DdGeom &d = dd->d;
    for (int i = 0; i < 4; i++) d.g[i] = gdims[i];
    d.t0 = t0;
    d.lt = lt;
    d.Vs = (uint32_t)gdims[0] * gdims[1] * gdims[2];
    d.F = d.Vs / 2;
    const size_t V = (size_t)d.Vs * gdims[3], Vloc = (size_t)d.Vs * lt;
    const size_t gbytes = 4 * V * 18 * sizeof(double), lbytes = 4 * Vloc * 18 * sizeof(double);
    double *gf = nullptr, *gl = nullptr, *lf = nullptr, *ll = nullptr;
    const double *sf = fat, *sl = lng;
    int rc = HISQ_OK;
    cudaError_t e = cudaSetDevice(opts.device);
    if (e == cudaSuccess && !opts.links_on_device) {
        e = cudaMalloc(&gf, gbytes);
        if (e == cudaSuccess) e = cudaMalloc(&gl, gbytes);
        if (e == cudaSuccess) e = cudaMemcpy(gf, fat, gbytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(gl, lng, gbytes, cudaMemcpyHostToDevice);
        sf = gf;
        sl = gl;
    }
    if (e == cudaSuccess) e = cudaMalloc(&lf, lbytes);
    if (e == cudaSuccess) e = cudaMalloc(&ll, lbytes);
    if (e == cudaSuccess) e = cudaMalloc(&dd->halo_links, 2 * 3 * (size_t)d.Vs * 18 * sizeof(double));
    if (e == cudaSuccess) {
        k_dd_slab_links<<<dim3((unsigned)((Vloc + 255) / 256), 4), 256>>>(d, sf, sl, lf, ll);
        k_dd_halo_links<<<dim3((d.Vs + 255) / 256, 3), 256>>>(d, sf, sl, dd->halo_links);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        rc = e == cudaErrorMemoryAllocation ? HISQ_ENOMEM : HISQ_ECUDA;
        dd_fail(dd, rc, std::string("hisq_dd_create: ") + cudaGetErrorString(e));
    } else {
        hisq_opts so;
        hisq_opts_default(&so);
        so.links_on_device = 1;
        so.links_phased = 1;
        so.prec_mask = 1u << HISQ_F64;
        so.device = opts.device;
        so.autotune = 0;
        const int ldims[4] = {gdims[0], gdims[1], gdims[2], lt};
        rc = hisq_create(&dd->slab, ldims, lf, ll, &so);
        if (rc) dd_fail(dd, rc, "hisq_dd_create: slab link store");
    }
    if (gf) cudaFree(gf);
    if (gl) cudaFree(gl);
    if (lf) cudaFree(lf);
    if (ll) cudaFree(ll);
    if (rc) {
        hisq_dd_destroy(dd);
        return rc;
    }
    *out = dd;
    return HISQ_OK;
}

int hisq_dd_pack(hisq_dd *dd, const double *in, double *send_lo, double *send_hi, void *stream)
{
    if (!dd) return HISQ_EINVAL;
    if (!in || !send_lo || !send_hi) return dd_fail(dd, HISQ_EINVAL, "hisq_dd_pack: bad argument");
    cudaError_t e = cudaSetDevice(dd->device);
    const size_t face = 3 * (size_t)dd->d.F * 48; // three slices of one parity
    const char *src = reinterpret_cast<const char *>(in);
    cudaStream_t st = (cudaStream_t)stream;
    if (e == cudaSuccess) e = cudaMemcpyAsync(send_lo, src, face, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(send_hi, src + (size_t)(dd->d.lt - 3) * dd->d.F * 48, face, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return dd_fail(dd, HISQ_ECUDA, std::string("hisq_dd_pack: ") + cudaGetErrorString(e));
    return HISQ_OK;
}

int hisq_dd_dslash(hisq_dd *dd, int out_parity, const double *in, const double *halo_lo, const double *halo_hi,
                   double *out, void *stream)
{
    if (!dd) return HISQ_EINVAL;
    if (!in || !halo_lo || !halo_hi || !out || (out_parity != 0 && out_parity != 1))
        return dd_fail(dd, HISQ_EINVAL, "hisq_dd_dslash: bad argument");
    const size_t Vh = (size_t)dd->d.Vs * dd->d.lt / 2, hb = 3 * (size_t)dd->d.F * 48;
    const char *o = reinterpret_cast<const char *>(out);
    auto overlaps = [&](const void *p, size_t n) {
        const char *x = static_cast<const char *>(p);
        return x < o + Vh * 48 && o < x + n;
    };
    if (overlaps(in, Vh * 48) || overlaps(halo_lo, hb) || overlaps(halo_hi, hb))
        return dd_fail(dd, HISQ_EINVAL, "hisq_dd_dslash: out overlaps an input");
    cudaError_t e = cudaSetDevice(dd->device);
    if (e != cudaSuccess) return dd_fail(dd, HISQ_ECUDA, cudaGetErrorString(e));
    const LinkStore &L = dd->slab->links[HISQ_F64];
    DdArgs a{};
    a.g = dd->slab->g;
    a.p = out_parity;
    a.links = L.base;
    a.slot_bytes = L.slot_bytes;
    a.halo_links = dd->halo_links;
    a.in = reinterpret_cast<const char *>(in);
    a.lo = reinterpret_cast<const char *>(halo_lo);
    a.hi = reinterpret_cast<const char *>(halo_hi);
    a.out = reinterpret_cast<char *>(out);
    a.F = dd->d.F;
    a.Vs = dd->d.Vs;
    k_dd_dslash<<<(unsigned)((Vh + 127) / 128), 128, 0, (cudaStream_t)stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return dd_fail(dd, HISQ_ECUDA, std::string("hisq_dd_dslash: ") + cudaGetErrorString(e));
    return HISQ_OK;
}

}  // extern "C"
