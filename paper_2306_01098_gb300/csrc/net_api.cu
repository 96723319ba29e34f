// net_api.cu -- C entry points of the learned preconditioner: network creation, weights,
// inference, loss gradient, training (Adam), persistence, and flexible CG with K = network.
#include <algorithm>
#include <chrono>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "blas.cuh"
#include "dslash.cuh"
#include "net.cuh"

namespace hisq {

int apply_mdagm(hisq_ctx *ctx, int prec, double m, const void *in, void *tmp, void *out, int nrhs, size_t rhs_bytes,
                cudaStream_t st, const Reduce *red, bool tune);

static int net_alloc(hisq_net *n, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_error(n->ctx, e, "network allocation");
    cudaMemset(*p, 0, bytes ? bytes : 16);
    n->allocs.push_back(*p);
    return HISQ_OK;
}

static void net_free(hisq_net *n)
{
    if (!n) return;
    for (void *p : n->allocs) cudaFree(p);
    n->allocs.clear();
    if (n->h_sc) cudaFreeHost(n->h_sc);
    if (n->st) cudaStreamDestroy(n->st);
    delete n;
}

static Reduce net_red(const hisq_net *n, int op, int nblocks, int ntotal)
{
    Reduce R;
    R.partials = n->partials;
    R.counter = n->counter;
    R.sc = n->sc;
    R.op = op;
    R.nblocks = nblocks;
    R.ntotal = ntotal;
    return R;
}

static int read_sc(hisq_net *n, cudaStream_t st)
{
    HISQ_CUDA(n->ctx, cudaMemcpyAsync(n->h_sc, n->sc, sizeof(Scalars) * 4, cudaMemcpyDeviceToHost, st));
    HISQ_CUDA(n->ctx, cudaStreamSynchronize(st));
    return HISQ_OK;
}

// initial weights: identity map, plus small seeded random hopping weights
static void init_weights(const hisq_net *n, std::vector<float> &w)
{
    std::mt19937_64 rng(n->opts.seed);
    std::normal_distribution<double> N(0.0, 1.0);
    w.assign(2 * (size_t)n->nw, 0.f);
    for (int l = 0; l < n->nlayer; l++) {
        const int cin = n->chans[l], cout = n->chans[l + 1];
        const double sd = n->opts.init_hop / std::sqrt((double)kNetTaps * cin);
        for (int tap = 0; tap < kNetTaps; tap++)
            for (int o = 0; o < cout; o++)
                for (int i = 0; i < cin; i++) {
                    const size_t q = 2 * ((size_t)n->woff[l] + ((size_t)tap * cout + o) * cin + i);
                    const double re = N(rng), im = N(rng);
                    if (tap == 0) {
                        w[q] = (o == i) ? 1.f : 0.f;
                    } else {
                        w[q] = (float)(sd * re);
                        w[q + 1] = (float)(sd * im);
                    }
                }
    }
}

// Adam on the real and imaginary parts of every weight (Kingma & Ba 2015)
__global__ void k_adam(float2 *w, const double2 *grad, float2 *m1, float2 *m2, int n, float lr, float b1, float b2,
                       float eps, int step)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    const float g[2] = {(float)grad[q].x, (float)grad[q].y};
    float *pw = reinterpret_cast<float *>(&w[q]);
    float *pm = reinterpret_cast<float *>(&m1[q]);
    float *pv = reinterpret_cast<float *>(&m2[q]);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        pm[k] = b1 * pm[k] + (1.f - b1) * g[k];
        pv[k] = b2 * pv[k] + (1.f - b2) * g[k] * g[k];
        pw[k] -= lr * (pm[k] / c1) / (sqrtf(pv[k] / c2) + eps);
    }
}

__global__ void k_loss_accum(const Scalars *sc, double *acc)
{
    *acc += sc[0].last / sc[1].last;
}

}  // namespace hisq

using namespace hisq;

extern "C" {

void hisq_net_opts_default(hisq_net_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->nlayer = 4;
    o->channels = 8;
    o->link_prec = HISQ_F16;
    o->epochs = 4;
    o->batch = 8;
    o->lr = 2e-3;
    o->beta1 = 0.9;
    o->beta2 = 0.999;
    o->eps = 1e-8;
    o->init_hop = 0.05;
    o->seed = 12345;
    o->tensor_cores = 1;
}

int hisq_net_create(hisq_ctx *ctx, const hisq_net_opts *opts_in, hisq_net **out)
{
    if (!ctx || !out) return HISQ_EINVAL;
    *out = nullptr;
    hisq_net_opts o;
    if (opts_in) o = *opts_in;
    else hisq_net_opts_default(&o);
    if (o.nlayer < 1 || o.nlayer > kNetMaxLayers || o.batch < 1 || o.epochs < 0 || !(o.lr > 0.0))
        return set_error(ctx, HISQ_EINVAL, "hisq_net_create: bad options");
    if (o.link_prec != HISQ_F32 && o.link_prec != HISQ_F16) return set_error(ctx, HISQ_EINVAL, "hisq_net_create: link precision");
    if (!ctx->links[o.link_prec].built || ctx->links[o.link_prec].nreal != 18)
        return set_error(ctx, HISQ_ENOTBUILT, "hisq_net_create: needs 18-real links of that precision");
    if (o.loss != 0 && o.loss != 1) return set_error(ctx, HISQ_EINVAL, "hisq_net_create: loss");
    if (o.loss == 1 && !(o.mass >= 0.0 && std::isfinite(o.mass)))
        return set_error(ctx, HISQ_EINVAL, "hisq_net_create: mass");
    if (o.loss == 1 && !ctx->links[HISQ_F64].built)
        return set_error(ctx, HISQ_ENOTBUILT, "hisq_net_create: the residual loss needs the FP64 links");
    hisq_net *n = new hisq_net();
    n->ctx = ctx;
    n->device = ctx->device;
    static std::atomic<unsigned long long> next_uid{1};
    n->uid = next_uid++;
    n->opts = o;
    n->nlayer = o.nlayer;
    n->link_prec = o.link_prec;
    n->chans[0] = n->chans[o.nlayer] = 1;
    for (int l = 1; l < o.nlayer; l++) n->chans[l] = o.channels;
    int nw = 0, maxc = 1;
    for (int l = 0; l < o.nlayer; l++) {
        if (!net_shape_supported(n->chans[l], n->chans[l + 1])) {
            delete n;
            return set_error(ctx, HISQ_EINVAL, "hisq_net_create: channel count must be 1, 2, 4 or 8");
        }
        n->woff[l] = nw;
        nw += kNetTaps * n->chans[l] * n->chans[l + 1];
        maxc = std::max(maxc, n->chans[l + 1]);
    }
    n->woff[o.nlayer] = nw;
    n->nw = nw;
    const size_t V = 2ull * ctx->g.Vh;
    const int nblocks = (int)((V + 127) / 128);
    n->nblk_vec = (int)std::min<size_t>((ctx->g.Vh + kVecBlock - 1) / kVecBlock, 4ull * ctx->sm_count);
    int rc = HISQ_OK;
    auto A = [&](void **p, size_t b) { if (rc == HISQ_OK) rc = net_alloc(n, p, b); };
    A((void **)&n->w, sizeof(float2) * nw);
    A((void **)&n->wadj, sizeof(float2) * kNetTaps * kNetMaxChan * kNetMaxChan);
    A((void **)&n->m1, sizeof(float2) * nw);
    A((void **)&n->m2, sizeof(float2) * nw);
    A((void **)&n->grad, sizeof(double2) * nw);
    for (int l = 0; l <= o.nlayer; l++) A((void **)&n->act[l], V * n->chans[l] * 12);
    A((void **)&n->gact[0], V * maxc * 12);
    A((void **)&n->gact[1], V * maxc * 12);
    A((void **)&n->part, sizeof(float2) * (size_t)nblocks * kNetTaps * kNetMaxChan * kNetMaxChan);
    A((void **)&n->partials, sizeof(double) * 8 * (size_t)std::max(n->nblk_vec, nblocks));
    A((void **)&n->counter, 64);
    A((void **)&n->sc, sizeof(Scalars) * 4);
    A((void **)&n->lossacc, sizeof(double));
    if (o.loss == 1)
        for (double **q : {&n->zb, &n->eb, &n->tb, &n->Aeb, &n->A2eb}) A((void **)q, (size_t)ctx->g.Vh * 48);
    if (rc) {
        net_free(n);
        return rc;
    }
    if (cudaMallocHost(&n->h_sc, sizeof(Scalars) * 4) != cudaSuccess ||
        cudaStreamCreateWithFlags(&n->st, cudaStreamNonBlocking) != cudaSuccess) {
        net_free(n);
        return set_error(ctx, HISQ_ENOMEM, "hisq_net_create: host resources");
    }
    std::vector<float> w;
    init_weights(n, w);
    cudaError_t e = cudaMemcpy(n->w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        net_free(n);
        return cuda_error(ctx, e, "hisq_net_create: weights");
    }
    *out = n;
    return HISQ_OK;
}

void hisq_net_destroy(hisq_net *n)
{
    if (!n) return;
    cudaSetDevice(n->device);
    cudaDeviceSynchronize();
    net_free(n);
}

long hisq_net_num_weights(const hisq_net *n) { return n ? n->nw : 0; }

int hisq_net_get_weights(const hisq_net *n, double *w)
{
    if (!n || !w) return HISQ_EINVAL;
    std::vector<float2> h(n->nw);
    HISQ_CUDA(n->ctx, cudaMemcpy(h.data(), n->w, sizeof(float2) * n->nw, cudaMemcpyDeviceToHost));
    for (int i = 0; i < n->nw; i++) {
        w[2 * i] = h[i].x;
        w[2 * i + 1] = h[i].y;
    }
    return HISQ_OK;
}

int hisq_net_set_weights(hisq_net *n, const double *w)
{
    if (!n || !w) return HISQ_EINVAL;
    std::vector<float2> h(n->nw);
    for (int i = 0; i < n->nw; i++) h[i] = make_float2((float)w[2 * i], (float)w[2 * i + 1]);
    HISQ_CUDA(n->ctx, cudaMemcpy(n->w, h.data(), sizeof(float2) * n->nw, cudaMemcpyHostToDevice));
    return HISQ_OK;
}

int hisq_net_apply(hisq_net *n, const double *b, double *z, void *stream)
{
    if (!n || !b || !z) return HISQ_EINVAL;
    return net_forward(n, b, z, (cudaStream_t)stream);
}

int hisq_net_loss_grad(hisq_net *n, const double *b, const double *x, double *loss, double *grad)
{
    if (!n || !b || !x) return HISQ_EINVAL;
    cudaStream_t st = n->st;
    HISQ_CUDA(n->ctx, cudaMemsetAsync(n->grad, 0, sizeof(double2) * n->nw, st));
    int rc = net_accumulate(n, b, x, 1.0, st);
    if (rc) return rc;
    if ((rc = read_sc(n, st))) return rc;
    if (loss) *loss = n->h_sc[0].last / n->h_sc[1].last;
    if (grad) HISQ_CUDA(n->ctx, cudaMemcpy(grad, n->grad, sizeof(double2) * n->nw, cudaMemcpyDeviceToHost));
    return check_device_status(n->ctx, st);
}

int hisq_net_train(hisq_net *n, int npairs, const double *B, const double *X, double *losses)
{
    if (!n || npairs < 1 || !B || !X) return HISQ_EINVAL;
    hisq_ctx *ctx = n->ctx;
    cudaStream_t st = n->st;
    const uint32_t Vh = ctx->g.Vh;
    const size_t vec = (size_t)Vh * 6; // doubles per vector
    // the scale of A^-1 seen by the data: <b,x>/<b,b> averaged over the first pairs
    double ratio = 0.0;
    const int nprobe = std::min(npairs, 8);
    for (int i = 0; i < nprobe; i++) {
        const double *b = B + i * vec, *x = X + i * vec;
        const dim3 g(n->nblk_vec, 1);
        k_cdot<HISQ_F64><<<g, kVecBlock, 0, st>>>(VecRef{(char *)b, 0}, VecRef{(char *)x, 0}, Vh,
                                                  net_red(n, FIN_CDOT, n->nblk_vec, n->nblk_vec));
        int rc = read_sc(n, st);
        if (rc) return rc;
        const double bx = n->h_sc[0].last;
        k_norm_f64<<<g, kVecBlock, 0, st>>>(VecRef{(char *)b, 0}, Vh, net_red(n, FIN_STORE, n->nblk_vec, n->nblk_vec));
        if ((rc = read_sc(n, st))) return rc;
        ratio += bx / n->h_sc[0].last;
    }
    ratio /= nprobe;
    const int last = n->nlayer - 1;
    const float2 s0 = make_float2((float)ratio, 0.f);
    HISQ_CUDA(ctx, cudaMemcpyAsync(n->w + n->woff[last], &s0, sizeof(float2), cudaMemcpyHostToDevice, st));
    std::vector<int> order(npairs);
    std::iota(order.begin(), order.end(), 0);
    std::mt19937_64 rng(n->opts.seed ^ 0x5bd1e995ull);
    const int bs = n->opts.batch;
    for (int ep = 0; ep < n->opts.epochs; ep++) {
        std::shuffle(order.begin(), order.end(), rng);
        HISQ_CUDA(ctx, cudaMemsetAsync(n->lossacc, 0, sizeof(double), st));
        for (int b0 = 0; b0 < npairs; b0 += bs) {
            const int nb = std::min(bs, npairs - b0);
            HISQ_CUDA(ctx, cudaMemsetAsync(n->grad, 0, sizeof(double2) * n->nw, st));
            for (int k = 0; k < nb; k++) {
                const int i = order[b0 + k];
                int rc = net_accumulate(n, B + i * vec, X + i * vec, 1.0 / nb, st);
                if (rc) return rc;
                k_loss_accum<<<1, 1, 0, st>>>(n->sc, n->lossacc);
            }
            n->step++;
            k_adam<<<(n->nw + 127) / 128, 128, 0, st>>>(n->w, n->grad, n->m1, n->m2, n->nw, (float)n->opts.lr,
                                                         (float)n->opts.beta1, (float)n->opts.beta2, (float)n->opts.eps,
                                                         n->step);
            HISQ_CUDA(ctx, cudaGetLastError());
        }
        double acc = 0.0;
        HISQ_CUDA(ctx, cudaMemcpyAsync(&acc, n->lossacc, sizeof(double), cudaMemcpyDeviceToHost, st));
        HISQ_CUDA(ctx, cudaStreamSynchronize(st));
        if (losses) losses[ep] = acc / npairs;
    }
    HISQ_CUDA(ctx, cudaStreamSynchronize(st));
    return check_device_status(ctx, st);
}

int hisq_net_save(const hisq_net *n, const char *path)
{
    if (!n || !path) return HISQ_EINVAL;
    std::vector<double> w(2 * (size_t)n->nw);
    int rc = hisq_net_get_weights(n, w.data());
    if (rc) return rc;
    FILE *f = std::fopen(path, "wb");
    if (!f) return set_error(n->ctx, HISQ_EINVAL, "hisq_net_save: cannot open file");
    const char magic[8] = {'H', 'I', 'S', 'Q', 'N', 'E', 'T', '1'};
    const int hdr[4] = {n->nlayer, n->opts.channels, n->link_prec, n->nw};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int), 4, f) == 4 &&
              std::fwrite(w.data(), sizeof(double), w.size(), f) == w.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? HISQ_OK : set_error(n->ctx, HISQ_EINVAL, "hisq_net_save: write failed");
}

int hisq_net_load(hisq_ctx *ctx, const char *path, hisq_net **out)
{
    if (!ctx || !path || !out) return HISQ_EINVAL;
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_error(ctx, HISQ_EINVAL, "hisq_net_load: cannot open file");
    char magic[8];
    int hdr[4];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "HISQNET1", 8) == 0 &&
              std::fread(hdr, sizeof(int), 4, f) == 4;
    hisq_net_opts o;
    hisq_net_opts_default(&o);
    std::vector<double> w;
    if (ok) {
        o.nlayer = hdr[0];
        o.channels = hdr[1];
        o.link_prec = hdr[2];
        w.resize(2 * (size_t)std::max(hdr[3], 0));
        ok = std::fread(w.data(), sizeof(double), w.size(), f) == w.size();
    }
    std::fclose(f);
    if (!ok) return set_error(ctx, HISQ_EINVAL, "hisq_net_load: bad file");
    int rc = hisq_net_create(ctx, &o, out);
    if (rc) return rc;
    if ((long)w.size() != 2 * (*out)->nw) {
        hisq_net_destroy(*out);
        *out = nullptr;
        return set_error(ctx, HISQ_EINVAL, "hisq_net_load: weight count mismatch");
    }
    return hisq_net_set_weights(*out, w.data());
}

}  // extern "C"

// hisq_net_create followed by hisq_net_train, the network returned only when both succeed
extern "C" int hisq_precond_train(hisq_ctx *ctx, const hisq_net_opts *opts, int npairs, const double *B,
                                  const double *X, hisq_net **net)
{
    if (!ctx) return HISQ_EINVAL;
    if (!net) return set_error(ctx, HISQ_EINVAL, "hisq_precond_train: bad argument");
    *net = nullptr;
    if (npairs < 1 || !B || !X) return set_error(ctx, HISQ_EINVAL, "hisq_precond_train: bad argument");
    hisq_net *n = nullptr;
    int rc = hisq_net_create(ctx, opts, &n);
    if (rc) return rc;
    rc = hisq_net_train(n, npairs, B, X, nullptr);
    if (rc) {
        hisq_net_destroy(n);
        return rc;
    }
    *net = n;
    return HISQ_OK;
}
