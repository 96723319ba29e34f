// context.cu -- context creation, link preparation and field conversion.
//
// Link preparation (one-time): canonical FP64 links [4][V][3][3] (Sec. 4.3 link index) are
// copied into one AoSoA store per requested precision.  For 18 reals the staggered phase
// eta_mu(x) and the antiperiodic time-boundary sign of the hop x -> x + k t^ (k = 1 for X,
// 3 for W) are multiplied into the link owned by x, so the kernels apply no signs.  For 12
// reals the first two rows of sign * L / c are kept, with c the real constant for which
// L / c is in SU(3) (one per link type, verified on every link); the kernels rebuild the
// third row and its sign.  16-bit stores keep L / s with s = max |entry| of the type.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "arith.cuh"
#include "dslash.cuh"

namespace hisq {

int set_error(hisq_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) {
        ctx->last_error = code;
        ctx->msg = msg;
    }
    return code;
}

int cuda_error(hisq_ctx *ctx, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return set_error(ctx, e == cudaErrorMemoryAllocation ? HISQ_ENOMEM : HISQ_ECUDA, m);
}

// Reads (and clears) the context's device error flag after the work queued on `st`:
// HISQ_EDEVICE with the recording site if a kernel raised it.
int check_device_status(hisq_ctx *ctx, cudaStream_t st)
{
    if (!ctx || !ctx->status) return HISQ_OK;
    DevStatus h{};
    cudaError_t e = cudaMemcpyAsync(&h, ctx->status, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(ctx, e, "device status");
    if (h.error == 0) return HISQ_OK;
    cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), st);
    cudaStreamSynchronize(st);
    return set_error(ctx, HISQ_EDEVICE,
                     h.where == 1 ? "a bounded wait of the tensor-core network layer ran out" : "device error flag raised");
}

int ensure_workspace(hisq_ctx *ctx, size_t bytes)
{
    if (ctx->ws_bytes >= bytes) return HISQ_OK;
    if (ctx->ws) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_error(ctx, e, "synchronise before workspace growth");
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    const size_t b = (bytes + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
    cudaError_t e = cudaMalloc(&ctx->ws, b);
    if (e != cudaSuccess) return cuda_error(ctx, e, "workspace allocation");
    ctx->ws_bytes = b;
    return HISQ_OK;
}

// ---------------------------------------------------------------- link conversion kernels
__device__ __forceinline__ void store_words(char *slot, uint32_t s, int LB, const uint32_t *w)
{
    const int NQ = LB / 16, TB = LB % 16;
    char *blk = slot + (size_t)(s >> 5) * (32 * LB);
    const uint32_t lane = s & 31;
    for (int q = 0; q < NQ; q++)
        *reinterpret_cast<uint4 *>(blk + q * 512 + lane * 16) = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    if (TB == 8) *reinterpret_cast<uint2 *>(blk + NQ * 512 + lane * 8) = make_uint2(w[4 * NQ], w[4 * NQ + 1]);
    if (TB == 4) *reinterpret_cast<uint32_t *>(blk + NQ * 512 + lane * 4) = w[4 * NQ];
}

struct ImportArgs {
    Geom g;
    const double *src[2]; // fat, long canonical [4][V][18]
    char *base;
    size_t slot_bytes;
    int prec, nreal, phased;
    double inv_scale[2];  // stored = sign * link * inv_scale
};

__global__ void k_import_links(const ImportArgs a)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    const int slot = blockIdx.y; // (p * 2 + type) * 4 + mu
    const int mu = slot & 3, type = (slot >> 2) & 1, p = slot >> 3;
    if (s >= a.g.VhPad) return;
    const int LB = link_bytes(a.prec, a.nreal);
    char *dst = a.base + (size_t)slot * a.slot_bytes;
    uint32_t w[36];
    for (int i = 0; i < 36; i++) w[i] = 0u;
    if (s < a.g.Vh) {
        const Site c = site_coords(a.g, s, p);
        const int k = type ? 3 : 1;
        int neg = 0;
        if (!a.phased) neg = eta_neg(c, mu) ^ ((mu == 3) && (c.t + k >= a.g.n[3]));
        const double sg = (neg ? -1.0 : 1.0) * a.inv_scale[type];
        const size_t V = 2ull * a.g.Vh;
        const double *L = a.src[type] + ((size_t)mu * V + (size_t)p * a.g.Vh + s) * 18;
        for (int i = 0; i < a.nreal; i++) {
            const double d = sg * L[i];
            switch (a.prec) {
            case HISQ_F64: {
                const unsigned long long b = __double_as_longlong(d);
                w[2 * i] = (uint32_t)b;
                w[2 * i + 1] = (uint32_t)(b >> 32);
                break;
            }
            case HISQ_F64X: {
                const float h = __double2float_rn(d);
                w[i] = __float_as_uint(h);
                w[a.nreal + i] = __float_as_uint(__double2float_rn(d - (double)h));
                break;
            }
            case HISQ_F32: w[i] = __float_as_uint(__double2float_rn(d)); break;
            case HISQ_F16: {
                const __half h = __double2half(d);
                const uint16_t u = *reinterpret_cast<const uint16_t *>(&h);
                w[i >> 1] |= (uint32_t)u << (16 * (i & 1));
                break;
            }
            default: {
                const __nv_bfloat16 h = __double2bfloat16(d);
                const uint16_t u = *reinterpret_cast<const uint16_t *>(&h);
                w[i >> 1] |= (uint32_t)u << (16 * (i & 1));
                break;
            }
            }
        }
    }
    store_words(dst, s, LB, w);
}

// max |entry| of each link type (for 16-bit scales) and, for a candidate c per type, the
// largest deviation of L / c from SU(3): max(|(L/c)^+ (L/c) - 1|, |det(L/c) - 1|)
struct LinkStats {
    unsigned int maxabs_bits[2];
    unsigned long long su3_err_bits[2];
};

__device__ __forceinline__ void cmul(double ar, double ai, double br, double bi, double &r, double &i)
{
    r = ar * br - ai * bi;
    i = ar * bi + ai * br;
}

__global__ void k_link_stats(const double *fat, const double *lng, size_t nlinks, double c0, double c1,
                             LinkStats *out)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const int type = blockIdx.y;
    if (i >= nlinks) return;
    const double *L = (type ? lng : fat) + i * 18;
    const double c = type ? c1 : c0;
    float m = 0.f;
    double u[18];
    for (int k = 0; k < 18; k++) {
        m = fmaxf(m, (float)fabs(L[k]));
        u[k] = L[k] / c;
    }
    atomicMax(&out->maxabs_bits[type], __float_as_uint(m));
    double err = 0.0;
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++) {
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < 3; k++) { // (U^+ U)_{rq} = sum_k conj(U_kr) U_kq
                double pr, pi;
                cmul(u[2 * (3 * k + r)], -u[2 * (3 * k + r) + 1], u[2 * (3 * k + q)], u[2 * (3 * k + q) + 1], pr, pi);
                sr += pr;
                si += pi;
            }
            err = fmax(err, fabs(sr - (r == q ? 1.0 : 0.0)) + fabs(si));
        }
    // det = row0 . (row1 x row2)
    double dr = 0.0, di = 0.0;
    for (int k = 0; k < 3; k++) {
        const int a = (k + 1) % 3, b = (k + 2) % 3;
        double xr, xi, yr, yi;
        cmul(u[6 + 2 * a], u[6 + 2 * a + 1], u[12 + 2 * b], u[12 + 2 * b + 1], xr, xi);
        cmul(u[6 + 2 * b], u[6 + 2 * b + 1], u[12 + 2 * a], u[12 + 2 * a + 1], yr, yi);
        double pr, pi;
        cmul(u[2 * k], u[2 * k + 1], xr - yr, xi - yi, pr, pi);
        dr += pr;
        di += pi;
    }
    err = fmax(err, fabs(dr - 1.0) + fabs(di));
    atomicMax(&out->su3_err_bits[type], (unsigned long long)__double_as_longlong(err));
}

// ---------------------------------------------------------------- field conversion kernels
template <int P>
__global__ void k_field_import(const double *src, char *dst, uint32_t Vh, size_t rhs_bytes, int nrhs)
{
    using T = Prec<P>;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (s >= Vh || r >= nrhs) return;
    const double *x = src + ((size_t)r * Vh + s) * 6;
    typename T::Acc a;
    T::zero(a);
    for (int i = 0; i < 6; i++) T::set_acc(a, i, x[i]);
    T::store(dst + (size_t)r * rhs_bytes, s, a);
}

template <int P>
__global__ void k_field_export(const char *src, double *dst, uint32_t Vh, size_t rhs_bytes, int nrhs)
{
    using T = Prec<P>;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (s >= Vh || r >= nrhs) return;
    typename T::Vec v;
    T::load(src + (size_t)r * rhs_bytes, s, v);
    double *x = dst + ((size_t)r * Vh + s) * 6;
    for (int i = 0; i < 6; i++) x[i] = T::vcomp(v, i);
}

int launch_import(hisq_ctx *ctx, int prec, const double *src, void *dst, int nrhs, size_t rhs_bytes, cudaStream_t st)
{
    dim3 grid((ctx->g.Vh + 255) / 256, nrhs);
    char *d = static_cast<char *>(dst);
    switch (prec) {
    case HISQ_F64: k_field_import<HISQ_F64><<<grid, 256, 0, st>>>(src, d, ctx->g.Vh, rhs_bytes, nrhs); break;
    case HISQ_F64X: k_field_import<HISQ_F64X><<<grid, 256, 0, st>>>(src, d, ctx->g.Vh, rhs_bytes, nrhs); break;
    case HISQ_F32: k_field_import<HISQ_F32><<<grid, 256, 0, st>>>(src, d, ctx->g.Vh, rhs_bytes, nrhs); break;
    case HISQ_F16: k_field_import<HISQ_F16><<<grid, 256, 0, st>>>(src, d, ctx->g.Vh, rhs_bytes, nrhs); break;
    case HISQ_BF16: k_field_import<HISQ_BF16><<<grid, 256, 0, st>>>(src, d, ctx->g.Vh, rhs_bytes, nrhs); break;
    default: return set_error(ctx, HISQ_EINVAL, "unknown precision");
    }
    HISQ_CUDA(ctx, cudaGetLastError());
    return HISQ_OK;
}

int launch_export(hisq_ctx *ctx, int prec, const void *src, double *dst, int nrhs, size_t rhs_bytes, cudaStream_t st)
{
    dim3 grid((ctx->g.Vh + 255) / 256, nrhs);
    const char *s = static_cast<const char *>(src);
    switch (prec) {
    case HISQ_F64: k_field_export<HISQ_F64><<<grid, 256, 0, st>>>(s, dst, ctx->g.Vh, rhs_bytes, nrhs); break;
    case HISQ_F64X: k_field_export<HISQ_F64X><<<grid, 256, 0, st>>>(s, dst, ctx->g.Vh, rhs_bytes, nrhs); break;
    case HISQ_F32: k_field_export<HISQ_F32><<<grid, 256, 0, st>>>(s, dst, ctx->g.Vh, rhs_bytes, nrhs); break;
    case HISQ_F16: k_field_export<HISQ_F16><<<grid, 256, 0, st>>>(s, dst, ctx->g.Vh, rhs_bytes, nrhs); break;
    case HISQ_BF16: k_field_export<HISQ_BF16><<<grid, 256, 0, st>>>(s, dst, ctx->g.Vh, rhs_bytes, nrhs); break;
    default: return set_error(ctx, HISQ_EINVAL, "unknown precision");
    }
    HISQ_CUDA(ctx, cudaGetLastError());
    return HISQ_OK;
}

// ---------------------------------------------------------------- context setup
static int build_store(hisq_ctx *ctx, int prec, int nreal, const double *fat, const double *lng, double c[2],
                       const LinkStats &stats)
{
    LinkStore &L = ctx->links[prec];
    const int LB = link_bytes(prec, nreal);
    L.nreal = nreal;
    L.slot_bytes = (size_t)ctx->g.VhPad * LB;
    cudaError_t e = cudaMalloc((void **)&L.base, L.slot_bytes * kSlots);
    if (e != cudaSuccess) return cuda_error(ctx, e, "link store allocation");
    ImportArgs a{};
    a.g = ctx->g;
    a.src[0] = fat;
    a.src[1] = lng;
    a.base = L.base;
    a.slot_bytes = L.slot_bytes;
    a.prec = prec;
    a.nreal = nreal;
    a.phased = ctx->links_phased;
    for (int t = 0; t < 2; t++) {
        double sc = 1.0;
        if (nreal == 12) sc = c[t];
        else if (prec == HISQ_F16 || prec == HISQ_BF16) {
            unsigned bits = stats.maxabs_bits[t];
            float m;
            std::memcpy(&m, &bits, 4);
            sc = m > 0.f ? (double)m : 1.0;
        }
        L.scale[t] = sc;
        a.inv_scale[t] = 1.0 / sc;
    }
    dim3 grid((ctx->g.VhPad + 127) / 128, kSlots);
    k_import_links<<<grid, 128>>>(a);
    HISQ_CUDA(ctx, cudaGetLastError());
    L.built = 1;
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" {

void hisq_opts_default(hisq_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->prec_mask = (1u << HISQ_F64) | (1u << HISQ_F64X) | (1u << HISQ_F32) | (1u << HISQ_F16);
    for (int i = 0; i < HISQ_NPREC; i++) o->compression[i] = 18;
    o->autotune = 1;
}

const char *hisq_strerror(int s)
{
    switch (s) {
    case HISQ_OK: return "ok";
    case HISQ_EINVAL: return "invalid argument";
    case HISQ_ENOMEM: return "out of memory";
    case HISQ_ECUDA: return "CUDA error";
    case HISQ_ENOTCONVERGED: return "solver did not converge";
    case HISQ_ETIMEOUT: return "device wait timed out";
    case HISQ_EDEVICE: return "device error flag raised";
    case HISQ_ENOTBUILT: return "precision or compression not built in this context";
    }
    return "unknown status";
}

int hisq_get_last_error(const hisq_ctx *ctx) { return ctx ? ctx->last_error : HISQ_EINVAL; }
const char *hisq_last_error_message(const hisq_ctx *ctx) { return ctx ? ctx->msg.c_str() : "null context"; }
long hisq_half_volume(const hisq_ctx *ctx) { return ctx ? (long)ctx->g.Vh : 0; }

void hisq_destroy(hisq_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    release_work(ctx);
    release_ms_work(ctx);
    release_fcg_work(ctx);
    for (auto &L : ctx->links)
        if (L.base) cudaFree(L.base);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->status) cudaFree(ctx->status);
    delete ctx;
}

int hisq_create(hisq_ctx **out, const int dims[4], const double *fat, const double *lng, const hisq_opts *opts_in)
{
    if (!out) return HISQ_EINVAL;
    *out = nullptr;
    if (!dims || !fat || !lng) return HISQ_EINVAL;
    hisq_opts opts;
    if (opts_in) opts = *opts_in;
    else hisq_opts_default(&opts);
    if (opts.prec_mask == 0) {
        hisq_opts d;
        hisq_opts_default(&d);
        opts.prec_mask = d.prec_mask;
    }
    for (int i = 0; i < 4; i++)
        if (dims[i] < 4 || (dims[i] & 1)) return HISQ_EINVAL;
    const unsigned long long V = (unsigned long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V / 2 >= (1ull << 30)) return HISQ_EINVAL;
    for (int p = 0; p < HISQ_NPREC; p++) {
        int c = opts.compression[p] == 0 ? 18 : opts.compression[p];
        if (c != 18 && c != 12) return HISQ_EINVAL;
        if (c == 12 && ((opts.prec_mask >> p) & 1) && (p == HISQ_F64X || opts.links_phased)) return HISQ_EINVAL;
        opts.compression[p] = c;
    }

    hisq_ctx *ctx = new hisq_ctx();
    ctx->device = opts.device;
    ctx->links_phased = opts.links_phased;
    ctx->autotune = opts.autotune;
    for (int i = 0; i < 4; i++) ctx->dims[i] = dims[i];
    cudaError_t e = cudaSetDevice(opts.device);
    if (e != cudaSuccess) {
        delete ctx;
        return HISQ_ECUDA;
    }
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, opts.device);
    {
        int maxp = 0;
        cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, opts.device);
        ctx->l2_persist_max = maxp > 0 ? (size_t)maxp : 0;
    }
    Geom &g = ctx->g;
    for (int i = 0; i < 4; i++) g.n[i] = dims[i];
    g.nxh = dims[0] / 2;
    g.Vh = (uint32_t)(V / 2);
    g.VhPad = (g.Vh + 127u) & ~127u;
    g.sy = g.nxh;
    g.sz = g.nxh * dims[1];
    g.st = g.nxh * dims[1] * dims[2];
    g.dx.init(g.nxh);
    g.dy.init(dims[1]);
    g.dz.init(dims[2]);
    g.dp.init(g.sz);
    g.dt.init(dims[3]);
    g.zt_ok = (g.sz % 32u) == 0 && dims[3] < dims[2];

    int rc = HISQ_OK;
    const size_t link_doubles = 4ull * V * 18;
    double *dfat = nullptr, *dlng = nullptr;
    bool own = !opts.links_on_device;
    LinkStats *dstats = nullptr;
    LinkStats stats{};
    double c[2] = {1.0, 1.0};
    bool need12 = false;
    for (int p = 0; p < HISQ_NPREC; p++)
        if (((opts.prec_mask >> p) & 1) && opts.compression[p] == 12) need12 = true;

    if (own) {
        e = cudaMalloc(&dfat, link_doubles * 8);
        if (e == cudaSuccess) e = cudaMalloc(&dlng, link_doubles * 8);
        if (e == cudaSuccess) e = cudaMemcpy(dfat, fat, link_doubles * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dlng, lng, link_doubles * 8, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            rc = cuda_error(ctx, e, "link upload");
            goto fail;
        }
    } else {
        dfat = const_cast<double *>(fat);
        dlng = const_cast<double *>(lng);
    }
    if (need12) {
        // c = real cube root of det of the first link of each type (checked on all links below)
        for (int t = 0; t < 2; t++) {
            double L[18];
            e = cudaMemcpy(L, t ? dlng : dfat, sizeof L, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { rc = cuda_error(ctx, e, "link read"); goto fail; }
            double dr = 0, di = 0;
            for (int k = 0; k < 3; k++) {
                const int a = (k + 1) % 3, b = (k + 2) % 3;
                const double xr = L[6 + 2 * a] * L[12 + 2 * b] - L[6 + 2 * a + 1] * L[12 + 2 * b + 1]
                                - (L[6 + 2 * b] * L[12 + 2 * a] - L[6 + 2 * b + 1] * L[12 + 2 * a + 1]);
                const double xi = L[6 + 2 * a] * L[12 + 2 * b + 1] + L[6 + 2 * a + 1] * L[12 + 2 * b]
                                - (L[6 + 2 * b] * L[12 + 2 * a + 1] + L[6 + 2 * b + 1] * L[12 + 2 * a]);
                dr += L[2 * k] * xr - L[2 * k + 1] * xi;
                di += L[2 * k] * xi + L[2 * k + 1] * xr;
            }
            if (std::fabs(di) > 1e-10 * std::fabs(dr) || dr == 0.0) {
                rc = set_error(ctx, HISQ_EINVAL, "12-real compression: link determinant is not real");
                goto fail;
            }
            c[t] = std::cbrt(dr);
        }
    }
    e = cudaMalloc(&dstats, sizeof(LinkStats));
    if (e == cudaSuccess) e = cudaMemset(dstats, 0, sizeof(LinkStats));
    if (e != cudaSuccess) { rc = cuda_error(ctx, e, "stats allocation"); goto fail; }
    {
        const size_t nl = 4ull * V;
        dim3 grid((unsigned)((nl + 255) / 256), 2);
        k_link_stats<<<grid, 256>>>(dfat, dlng, nl, c[0], c[1], dstats);
        e = cudaMemcpy(&stats, dstats, sizeof stats, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { rc = cuda_error(ctx, e, "link statistics"); goto fail; }
    }
    if (need12) {
        for (int t = 0; t < 2; t++) {
            double err;
            std::memcpy(&err, &stats.su3_err_bits[t], 8);
            if (!(err <= 1e-10)) {
                rc = set_error(ctx, HISQ_EINVAL, "12-real compression: links are not a constant times SU(3)");
                goto fail;
            }
        }
    }
    for (int p = 0; p < HISQ_NPREC && rc == HISQ_OK; p++)
        if ((opts.prec_mask >> p) & 1) rc = build_store(ctx, p, opts.compression[p], dfat, dlng, c, stats);
    if (rc != HISQ_OK) goto fail;
    e = cudaMalloc(&ctx->status, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { rc = cuda_error(ctx, e, "link preparation"); goto fail; }
    if (own) { cudaFree(dfat); cudaFree(dlng); }
    cudaFree(dstats);
    *out = ctx;
    return HISQ_OK;
fail:
    if (own) { cudaFree(dfat); cudaFree(dlng); }
    if (dstats) cudaFree(dstats);
    hisq_destroy(ctx);
    return rc;
}

// ---------------------------------------------------------------- fields
int hisq_field_create(hisq_ctx *ctx, int prec, int nrhs, hisq_field **f)
{
    if (!ctx || !f || prec < 0 || prec >= HISQ_NPREC || nrhs < 1) return set_error(ctx, HISQ_EINVAL, "field_create");
    *f = nullptr;
    hisq_field *x = new hisq_field();
    x->ctx = ctx;
    x->prec = prec;
    x->nrhs = nrhs;
    x->rhs_bytes = (size_t)ctx->g.VhPad * spinor_bytes(prec);
    cudaError_t e = cudaMalloc(&x->data, x->rhs_bytes * nrhs);
    if (e == cudaSuccess) e = cudaMemset(x->data, 0, x->rhs_bytes * nrhs);
    if (e != cudaSuccess) {
        delete x;
        return cuda_error(ctx, e, "field allocation");
    }
    *f = x;
    return HISQ_OK;
}

void hisq_field_destroy(hisq_field *f)
{
    if (!f) return;
    if (f->data) cudaFree(f->data);
    delete f;
}

size_t hisq_field_bytes(const hisq_field *f) { return f ? f->rhs_bytes * f->nrhs : 0; }

int hisq_field_import(hisq_field *f, const double *src, void *stream)
{
    if (!f || !src) return HISQ_EINVAL;
    return launch_import(f->ctx, f->prec, src, f->data, f->nrhs, f->rhs_bytes, (cudaStream_t)stream);
}

int hisq_field_export(const hisq_field *f, double *dst, void *stream)
{
    if (!f || !dst) return HISQ_EINVAL;
    return launch_export(f->ctx, f->prec, f->data, dst, f->nrhs, f->rhs_bytes, (cudaStream_t)stream);
}

}  // extern "C"
