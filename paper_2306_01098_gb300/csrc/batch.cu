// batch.cu -- lattices of different sizes in single launches: the batched Dslash and the
// batched CG (one system per lattice).
//
// A batch is an internal context whose Vh is the largest member's.  Its vectors hold the
// lattices as right-hand sides of that padded size (lattice k = right-hand side k, sites
// beyond its own half volume are zero and never written by the operator), so the solver
// of hisq_cg runs unchanged; only the Dslash differs: one launch covers the site tiles of
// every lattice, and each block reads the geometry and link store of its lattice from the
// batch table.  Lattice k's mass enters as the per-right-hand-side shift 4 m_k^2.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dslash.cuh"

namespace hisq {

int run_cg(hisq_ctx *ctx, double m, const double *b, double *x, int nrhs, const hisq_solve_opts &o, hisq_stats *stats,
           double *residuals, const double *shifts);
int launch_dslash2(hisq_ctx *ctx, int pl, int pv, int out_parity, const void *in, void *out, int nrhs, size_t rhs_bytes,
                   cudaStream_t st);
int launch_import(hisq_ctx *ctx, int prec, const double *src, void *dst, int nrhs, size_t rhs_bytes, cudaStream_t st);
int launch_export(hisq_ctx *ctx, int prec, const void *src, double *dst, int nrhs, size_t rhs_bytes, cudaStream_t st);

// packed canonical vectors (lattice k from site offset off[k], vh[k] sites, 6 doubles per
// site) <-> padded canonical vectors ([n][vhmax] sites, zero beyond vh[k])
__global__ void k_batch_pack(const double *src, double *dst, const unsigned long long *off, const uint32_t *vh,
                             uint32_t vhmax)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; // double within lattice
    const int k = blockIdx.y;
    if (e >= (size_t)vhmax * 6) return;
    dst[(size_t)k * vhmax * 6 + e] = e < (size_t)vh[k] * 6 ? src[off[k] * 6 + e] : 0.0;
}

__global__ void k_batch_unpack(const double *src, double *dst, const unsigned long long *off, const uint32_t *vh,
                               uint32_t vhmax)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (e >= (size_t)vh[k] * 6) return;
    dst[off[k] * 6 + e] = src[(size_t)k * vhmax * 6 + e];
}

}  // namespace hisq

using namespace hisq;

struct hisq_batch {
    hisq_ctx *v = nullptr; // the batch context
    int n = 0;
    std::vector<hisq_ctx *> members;
    size_t total = 0;                 // sum of the members' half volumes
    unsigned long long *d_off = nullptr; // packed site offsets (device)
    uint32_t *d_vh = nullptr;         // half volumes (device)
    double *pad_in = nullptr, *pad_out = nullptr; // padded canonical FP64 [n][vhmax]
};

static void batch_free(hisq_batch *b)
{
    if (!b) return;
    if (b->v) {
        hisq_ctx *v = b->v;
        cudaSetDevice(v->device);
        cudaDeviceSynchronize();
        release_work(v);
        release_ms_work(v);
        release_fcg_work(v);
        if (v->ws) cudaFree(v->ws);
        if (v->batch) cudaFree(v->batch);
        delete v->batch_host;
        delete v;
    }
    if (b->d_off) cudaFree(b->d_off);
    if (b->d_vh) cudaFree(b->d_vh);
    if (b->pad_in) cudaFree(b->pad_in);
    if (b->pad_out) cudaFree(b->pad_out);
    delete b;
}

static int pack(hisq_batch *b, const double *src, double *dst, cudaStream_t st)
{
    const uint32_t vhmax = b->v->g.Vh;
    dim3 grid((unsigned)(((size_t)vhmax * 6 + 255) / 256), b->n);
    k_batch_pack<<<grid, 256, 0, st>>>(src, dst, b->d_off, b->d_vh, vhmax);
    HISQ_CUDA(b->v, cudaGetLastError());
    return HISQ_OK;
}

static int unpack(hisq_batch *b, const double *src, double *dst, cudaStream_t st)
{
    const uint32_t vhmax = b->v->g.Vh;
    dim3 grid((unsigned)(((size_t)vhmax * 6 + 255) / 256), b->n);
    k_batch_unpack<<<grid, 256, 0, st>>>(src, dst, b->d_off, b->d_vh, vhmax);
    HISQ_CUDA(b->v, cudaGetLastError());
    return HISQ_OK;
}

extern "C" {

int hisq_batch_create(hisq_batch **out, int n, hisq_ctx *const *ctxs)
{
    if (!out) return HISQ_EINVAL;
    *out = nullptr;
    if (n < 1 || n > kMaxBatch || !ctxs) return HISQ_EINVAL;
    for (int k = 0; k < n; k++)
        if (!ctxs[k] || ctxs[k]->batch || ctxs[k]->device != ctxs[0]->device) return HISQ_EINVAL;
    hisq_batch *b = new hisq_batch();
    b->n = n;
    b->members.assign(ctxs, ctxs + n);
    hisq_ctx *v = new hisq_ctx();
    b->v = v;
    const hisq_ctx &c0 = *ctxs[0];
    v->device = c0.device;
    v->sm_count = c0.sm_count;
    v->l2_persist_max = c0.l2_persist_max;
    v->autotune = 1;
    BatchDesc *h = new BatchDesc();
    v->batch_host = h;
    h->n = n;
    uint32_t vhmax = 0;
    std::vector<unsigned long long> off(n);
    std::vector<uint32_t> vh(n);
    for (int k = 0; k < n; k++) {
        const hisq_ctx &c = *ctxs[k];
        vhmax = std::max(vhmax, c.g.Vh);
        off[k] = b->total;
        vh[k] = c.g.Vh;
        b->total += c.g.Vh;
        h->vh[k] = c.g.Vh;
        v->autotune &= c.autotune;
        BatchLattice &L = h->lat[k];
        L.g = c.g;
        for (int p = 0; p < HISQ_NPREC; p++) {
            L.links[p] = c.links[p].base;
            L.slot_bytes[p] = c.links[p].slot_bytes;
            L.scale[p][0] = c.links[p].scale[0];
            L.scale[p][1] = c.links[p].scale[1];
            L.scale_f[p][0] = (float)c.links[p].scale[0];
            L.scale_f[p][1] = (float)c.links[p].scale[1];
        }
    }
    for (int d = 0; d < 3; d++) {
        const size_t ds = (size_t)1 << d;
        size_t acc = 0, mx = 0;
        for (int k = 0; k < n; k++) {
            h->tstart[d][k] = (uint32_t)acc;
            const size_t t = ((size_t)vh[k] * ds + kDslashBlock - 1) / kDslashBlock;
            acc += t;
            mx = std::max(mx, t);
        }
        h->tstart[d][n] = (uint32_t)acc;
        h->maxtiles[d] = (uint32_t)mx;
    }
    // a precision is available when every member built it with the same compression
    for (int p = 0; p < HISQ_NPREC; p++) {
        bool all = true;
        for (int k = 0; k < n; k++)
            all &= ctxs[k]->links[p].built && ctxs[k]->links[p].nreal == c0.links[p].nreal;
        v->links[p].built = all;
        v->links[p].nreal = c0.links[p].nreal;
    }
    Geom &g = v->g;
    g.Vh = vhmax;
    g.VhPad = (vhmax + 127u) & ~127u;
    g.zt_ok = 0;
    int rc = HISQ_OK;
    cudaError_t e = cudaSetDevice(v->device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&v->batch, sizeof(BatchDesc));
    if (e == cudaSuccess) e = cudaMemcpy(v->batch, h, sizeof(BatchDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_off, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_off, off.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_vh, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_vh, vh.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice);
    const size_t pb = (size_t)n * vhmax * 48;
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->pad_in, pb);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->pad_out, pb);
    if (e == cudaSuccess) e = cudaMemset(b->pad_in, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(b->pad_out, 0, pb);
    if (e != cudaSuccess) {
        rc = e == cudaErrorMemoryAllocation ? HISQ_ENOMEM : HISQ_ECUDA;
        cudaGetLastError();
        batch_free(b);
        return rc;
    }
    *out = b;
    return HISQ_OK;
}

void hisq_batch_destroy(hisq_batch *b) { batch_free(b); }

long hisq_batch_sites(const hisq_batch *b) { return b ? (long)b->total : 0; }

const char *hisq_batch_last_error_message(hisq_batch *b) { return b ? b->v->msg.c_str() : ""; }

int hisq_batch_dslash(hisq_batch *b, int out_parity, const double *in, double *out, int prec, void *stream)
{
    if (!b) return HISQ_EINVAL;
    hisq_ctx *v = b->v;
    if (!in || !out || (out_parity != 0 && out_parity != 1) || prec < 0 || prec >= HISQ_NPREC)
        return set_error(v, HISQ_EINVAL, "hisq_batch_dslash: bad argument");
    if (!v->links[prec].built) return set_error(v, HISQ_ENOTBUILT, "hisq_batch_dslash: precision not built");
    cudaStream_t st = (cudaStream_t)stream;
    HISQ_CUDA(v, cudaSetDevice(v->device));
    int rc;
    if ((rc = pack(b, in, b->pad_in, st))) return rc;
    const int n = b->n;
    if (prec == HISQ_F64) {
        if ((rc = launch_dslash2(v, HISQ_F64, HISQ_F64, out_parity, b->pad_in, b->pad_out, n, (size_t)v->g.Vh * 48, st)))
            return rc;
    } else {
        const int pv = vector_prec(prec);
        const size_t rb = (size_t)v->g.VhPad * spinor_bytes(pv);
        if ((rc = ensure_workspace(v, 2 * rb * n))) return rc;
        char *t_in = static_cast<char *>(v->ws), *t_out = t_in + rb * n;
        if ((rc = launch_import(v, pv, b->pad_in, t_in, n, rb, st))) return rc;
        if ((rc = launch_dslash2(v, prec, pv, out_parity, t_in, t_out, n, rb, st))) return rc;
        if ((rc = launch_export(v, pv, t_out, b->pad_out, n, rb, st))) return rc;
    }
    return unpack(b, b->pad_out, out, st);
}

int hisq_batch_cg(hisq_batch *b, const double *m, const double *bvec, double *x, const hisq_solve_opts *opts,
                  hisq_stats *stats, double *residuals)
{
    if (!b) return HISQ_EINVAL;
    hisq_ctx *v = b->v;
    if (!m || !bvec || !x) return set_error(v, HISQ_EINVAL, "hisq_batch_cg: bad argument");
    hisq_solve_opts o;
    if (opts) o = *opts;
    else hisq_solve_opts_default(&o);
    if (o.host_buffers) return set_error(v, HISQ_EINVAL, "hisq_batch_cg: device buffers only");
    std::vector<double> shifts(b->n);
    for (int k = 0; k < b->n; k++) {
        if (!(m[k] >= 0.0) || !std::isfinite(m[k])) return set_error(v, HISQ_EINVAL, "hisq_batch_cg: bad mass");
        shifts[k] = 4.0 * m[k] * m[k];
    }
    HISQ_CUDA(v, cudaSetDevice(v->device));
    cudaStream_t st = (cudaStream_t)o.stream;
    int rc;
    if ((rc = pack(b, bvec, b->pad_in, st))) return rc;
    if (!o.zero_guess && (rc = pack(b, x, b->pad_out, st))) return rc;
    rc = run_cg(v, 0.0, b->pad_in, b->pad_out, b->n, o, stats, residuals, shifts.data());
    if (rc != HISQ_OK && rc != HISQ_ENOTCONVERGED) return rc;
    const int rc2 = unpack(b, b->pad_out, x, st);
    return rc2 ? rc2 : rc;
}

}  // extern "C"
