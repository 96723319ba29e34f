// noalloc.cu -- the normal operator A = 4m^2 - D_eo D_oe in FP64 without any device allocation.
//
// hisq_mdagm keeps its odd-parity intermediate (D_oe in) in a workspace that grows with
// cudaMalloc.  Some callers cannot let a library allocate: applications whose device memory
// is owned by another allocator or held to a fixed budget, and code that must not call
// cudaMalloc / cudaFree in its loop because those calls synchronise the whole device.  For
// them hisq_mdagm_noalloc keeps the intermediate in a fixed array in device memory instead.
//
// The array is a file-scope __device__ variable of kNoAllocScratchSites half-lattice sites
// (48 bytes each, 48 MiB in all).  Every GPU that loads this library's device code holds
// it until the process exits.  Host code only ever sees a host-side stand-in for the name,
// so the device address is looked up once per device with cudaGetSymbolAddress.
#include <mutex>

#include "dslash.cuh"

namespace hisq {

int apply_mdagm(hisq_ctx *ctx, int prec, double m, const void *in, void *tmp, void *out, int nrhs, size_t rhs_bytes,
                cudaStream_t st, const Reduce *red, bool tune);

constexpr size_t kNoAllocScratchSites = size_t(1) << 20; // nrhs * Vh must not exceed this
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchSites * 6];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[kNoAllocMaxDevices];

// device address of the scratch array on `dev`, which the caller has made current (looked
// up once per device, then cached)
static int noalloc_scratch(hisq_ctx *ctx, int dev, void **addr)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(ctx, HISQ_EINVAL, "hisq_mdagm_noalloc: device ordinal");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(ctx, e, "hisq_mdagm_noalloc: cudaGetSymbolAddress");
        g_noalloc_addr[dev] = p;
    }
    *addr = g_noalloc_addr[dev];
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_mdagm_noalloc(hisq_ctx *ctx, double m, const double *in, double *out, int nrhs, void *stream)
{
    if (!ctx) return HISQ_EINVAL;
    if (!in || !out || nrhs < 1) return set_error(ctx, HISQ_EINVAL, "hisq_mdagm_noalloc: bad argument");
    if (!ctx->links[HISQ_F64].built) return set_error(ctx, HISQ_ENOTBUILT, "hisq_mdagm_noalloc: FP64 links not built");
    const size_t sites = (size_t)nrhs * ctx->g.Vh;
    if (sites > kNoAllocScratchSites)
        return set_error(ctx, HISQ_EINVAL,
                         "hisq_mdagm_noalloc: nrhs * Vh exceeds the fixed scratch of 1048576 half-lattice sites");
    const size_t bytes = sites * 48;
    const char *a = reinterpret_cast<const char *>(in), *b = reinterpret_cast<const char *>(out);
    if (a < b + bytes && b < a + bytes) return set_error(ctx, HISQ_EINVAL, "hisq_mdagm_noalloc: in and out overlap");
    // the kernels run on the context's device, where its links and the scratch array live
    HISQ_CUDA(ctx, cudaSetDevice(ctx->device));
    void *scratch = nullptr;
    int rc = noalloc_scratch(ctx, ctx->device, &scratch);
    if (rc) return rc;
    // the intermediate covers every site of every right-hand side, so nothing needs clearing
    return apply_mdagm(ctx, HISQ_F64, m, in, scratch, out, nrhs, (size_t)ctx->g.Vh * 48, (cudaStream_t)stream,
                       nullptr, false);
}
