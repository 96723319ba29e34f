// net.cuh -- state of the learned preconditioner (gauge-covariant parallel-transport network).
#pragma once

#include <vector>

#include "internal.cuh"
#include "reduce.cuh"

namespace hisq {

constexpr int kNetTaps = 17;     // identity, 8 one-hop and 8 three-hop transports
constexpr int kNetMaxChan = 8;   // hidden complex channels
constexpr int kNetMaxLayers = 8;

bool net_shape_supported(int cin, int cout);

}  // namespace hisq

struct hisq_net {
    hisq_ctx *ctx = nullptr;
    int device = 0; // the context's device (teardown does not read the context)
    hisq_net_opts opts{};
    int nlayer = 0;
    int chans[hisq::kNetMaxLayers + 1] = {};
    int link_prec = HISQ_F32;
    int nw = 0;                                  // complex weights
    int woff[hisq::kNetMaxLayers + 1] = {};      // offset of each layer's block
    float2 *w = nullptr, *wadj = nullptr, *m1 = nullptr, *m2 = nullptr;
    double2 *grad = nullptr;
    uint32_t *act[hisq::kNetMaxLayers + 1] = {};
    uint32_t *gact[2] = {};
    float2 *part = nullptr;
    double *partials = nullptr;
    unsigned *counter = nullptr;
    hisq::Scalars *sc = nullptr, *h_sc = nullptr;
    double *lossacc = nullptr;
    double *zb = nullptr, *eb = nullptr, *tb = nullptr, *Aeb = nullptr, *A2eb = nullptr; // loss 1 (FP64)
    int nblk_vec = 0;
    int step = 0;
    unsigned long long uid = 0;                  // unique per network (keys cached solver graphs)
    cudaStream_t st = nullptr;
    std::vector<void *> allocs;
};

namespace hisq {
// reads and clears the context's device error flag (HISQ_EDEVICE if a kernel raised it)
int check_device_status(hisq_ctx *ctx, cudaStream_t st);
int net_forward(hisq_net *n, const double *b, double *z, cudaStream_t st);
int net_accumulate(hisq_net *n, const double *b, const double *x, double scale, cudaStream_t st);
}  // namespace hisq
