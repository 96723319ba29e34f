// net.cu -- gauge-covariant parallel-transport network (learned preconditioner; not in the
// paper) with its forward, backward and Adam kernels, and the training loop.
//
// Layer l maps C_in -> C_out complex channels on the full lattice:
//   psi'_{c'}(x) = sum_tap sum_c w[tap][c'][c] (T_tap psi_c)(x),
//   tap 0 = identity; tap 1+2mu+s = one hop, tap 9+2mu+s = three hops (s = 0 forward,
//   s = 1 backward) with the Dslash transports X_mu(x) psi(x+mu), X_mu(x-mu)^+ psi(x-mu),
//   W_mu(x) psi(x+3mu), W_mu(x-3mu)^+ psi(x-3mu) of the phased links (the context's link store,
//   where phases and the time boundary are folded in).  D itself is one such layer.
// The network K maps a source on even sites (odd sites zero) through the layers and keeps
// the even sites of the result.  Activations are stored in BF16 ([V][C][3 complex]),
// arithmetic and weights in FP32; gradients are reduced in FP64.
//   backward data:   g_in[c] = sum_tap sum_c' conj(w[tap][c'][c]) T_tap^+ g_out[c']
//                    (T^+ of a forward tap is the backward tap of the same direction and
//                    length, so the forward kernel runs with re-indexed conjugate weights)
//   backward weights: G[tap][c'][c] = sum_x sum_colour conj((T_tap psi_c)(x)) g_out[c'](x)
// Loss per (b, x) pair: |K(b) - x|^2 / |x|^2 on even sites.  Optimiser: Adam.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "arith.cuh"
#include "blas.cuh"
#include "net.cuh"
#include "tc.cuh"

namespace hisq {

int apply_mdagm(hisq_ctx *ctx, int prec, double m, const void *in, void *tmp, void *out, int nrhs, size_t rhs_bytes,
                cudaStream_t st, const Reduce *red, bool tune);

// ---------------------------------------------------------------- activation access
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint32_t bf_pack(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// channel c of site i: 3 complex numbers = 3 words
template <int C>
__device__ __forceinline__ void load_chan(const uint32_t *act, uint32_t i, int c, float (&v)[6])
{
    const uint32_t *p = act + ((size_t)i * C + c) * 3;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const uint32_t w = __ldg(p + k);
        v[2 * k] = bf_lo(w);
        v[2 * k + 1] = bf_hi(w);
    }
}

struct NetLayerArgs {
    Geom g;
    const char *links;
    size_t slot_bytes;
    float scale[2];
    const float2 *w;     // [17][cout][cin]
    const uint32_t *in;  // [V][cin][3] bf16 complex
    uint32_t *out;       // [V][cout][3]
    int even_only_in;    // input lives on even sites only (odd sites read as zero)
    int even_only_out;   // compute the even output sites only (the odd ones are not written)
    int tensor_cores;    // C -> C layers with C = 8 mix channels on the tensor cores
    int selftest_wait;   // first wait (bounded) on a barrier that nothing completes
    DevStatus *status;   // device error flag (bounded waits of the tensor-core layer)
};

template <int PL>
__device__ __forceinline__ void tap_link(const NetLayerArgs &a, const Site &c, uint32_t s, int p, int mu, int h,
                                         typename Prec<HISQ_F32>::Link &U, uint32_t &sn, bool &back, int &type)
{
    constexpr int LB = LinkBytes<PL>::b18;
    const int k = h == 0 ? 1 : h == 1 ? -1 : h == 2 ? 3 : -3;
    type = h >> 1;
    back = h & 1;
    bool wrap;
    sn = neighbour(a.g, c, s, mu, k, wrap);
    const int lp = back ? 1 - p : p;
    const char *slot = a.links + (size_t)((lp * 2 + type) * 4 + mu) * a.slot_bytes;
    uint32_t w[LB / 4];
    load_link_words<LB>(slot, back ? sn : s, w);
    Prec<PL>::template unpack<18>(w, U);
    if constexpr (PL == HISQ_F16 || PL == HISQ_BF16) {
        const float sc = a.scale[type];
#pragma unroll
        for (int q = 0; q < 18; q++) U.v[q] *= sc;
    }
}

__device__ __forceinline__ void transport(const typename Prec<HISQ_F32>::Link &U, bool dag, const float (&v)[6],
                                          float (&t)[6])
{
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float ur = dag ? U.v[2 * (3 * j + i)] : U.v[2 * (3 * i + j)];
            const float ui = dag ? -U.v[2 * (3 * j + i) + 1] : U.v[2 * (3 * i + j) + 1];
            re = fmaf(ur, v[2 * j], fmaf(-ui, v[2 * j + 1], re));
            im = fmaf(ur, v[2 * j + 1], fmaf(ui, v[2 * j], im));
        }
        t[2 * i] = re;
        t[2 * i + 1] = im;
    }
}

// forward layer (also the backward-data pass with re-indexed conjugate weights)
template <int PL, int CIN, int COUT>
__global__ void __launch_bounds__(128) k_net_layer(const NetLayerArgs a)
{
    __shared__ float2 sw[kNetTaps * COUT * CIN];
    for (int q = threadIdx.x; q < kNetTaps * COUT * CIN; q += blockDim.x) sw[q] = a.w[q];
    __syncthreads();
    // blocks alternate between the parities over the same range of half-sites, so the two
    // sites that use one link (its owner and the neighbour it reaches back from) run at
    // about the same time and the second use finds the link in L2
    const int p = a.even_only_out ? 0 : (int)(blockIdx.x & 1);
    const uint32_t s = (a.even_only_out ? blockIdx.x : blockIdx.x >> 1) * blockDim.x + threadIdx.x;
    if (s >= a.g.Vh) return;
    const uint32_t i = s + (uint32_t)p * a.g.Vh;
    float acc[COUT][6];
#pragma unroll
    for (int o = 0; o < COUT; o++)
#pragma unroll
        for (int k = 0; k < 6; k++) acc[o][k] = 0.f;
    // tap 0: identity
    if (!(a.even_only_in && p)) {
#pragma unroll
        for (int ci = 0; ci < CIN; ci++) {
            float v[6];
            load_chan<CIN>(a.in, i, ci, v);
#pragma unroll
            for (int o = 0; o < COUT; o++) {
                const float2 w = sw[o * CIN + ci];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    acc[o][2 * k] = fmaf(w.x, v[2 * k], fmaf(-w.y, v[2 * k + 1], acc[o][2 * k]));
                    acc[o][2 * k + 1] = fmaf(w.x, v[2 * k + 1], fmaf(w.y, v[2 * k], acc[o][2 * k + 1]));
                }
            }
        }
    }
    const Site c = site_coords(a.g, s, p);
    const bool nb_zero = a.even_only_in && (1 - p); // neighbours are odd: zero input
    if (!nb_zero) {
#pragma unroll 1
        for (int mu = 0; mu < 4; mu++) {
#pragma unroll
            for (int h = 0; h < 4; h++) {
                typename Prec<HISQ_F32>::Link U;
                uint32_t sn;
                bool back;
                int type;
                tap_link<PL>(a, c, s, p, mu, h, U, sn, back, type);
                const int tap = (type ? 9 : 1) + 2 * mu + (back ? 1 : 0);
                const uint32_t n = sn + (uint32_t)(1 - p) * a.g.Vh;
                if constexpr (COUT < CIN) {
                    // fewer outputs than inputs: mix the channels at the neighbour, then
                    // transport each output once (the transport is linear and colour-only)
                    float u[COUT][6];
#pragma unroll
                    for (int o = 0; o < COUT; o++)
#pragma unroll
                        for (int k = 0; k < 6; k++) u[o][k] = 0.f;
#pragma unroll
                    for (int ci = 0; ci < CIN; ci++) {
                        float v[6];
                        load_chan<CIN>(a.in, n, ci, v);
#pragma unroll
                        for (int o = 0; o < COUT; o++) {
                            const float2 w = sw[(tap * COUT + o) * CIN + ci];
#pragma unroll
                            for (int k = 0; k < 3; k++) {
                                u[o][2 * k] = fmaf(w.x, v[2 * k], fmaf(-w.y, v[2 * k + 1], u[o][2 * k]));
                                u[o][2 * k + 1] = fmaf(w.x, v[2 * k + 1], fmaf(w.y, v[2 * k], u[o][2 * k + 1]));
                            }
                        }
                    }
#pragma unroll
                    for (int o = 0; o < COUT; o++) {
                        float t[6];
                        transport(U, back, u[o], t);
#pragma unroll
                        for (int k = 0; k < 6; k++) acc[o][k] += t[k];
                    }
                } else {
#pragma unroll
                    for (int ci = 0; ci < CIN; ci++) {
                        float v[6], t[6];
                        load_chan<CIN>(a.in, n, ci, v);
                        transport(U, back, v, t);
#pragma unroll
                        for (int o = 0; o < COUT; o++) {
                            const float2 w = sw[(tap * COUT + o) * CIN + ci];
#pragma unroll
                            for (int k = 0; k < 3; k++) {
                                acc[o][2 * k] = fmaf(w.x, t[2 * k], fmaf(-w.y, t[2 * k + 1], acc[o][2 * k]));
                                acc[o][2 * k + 1] = fmaf(w.x, t[2 * k + 1], fmaf(w.y, t[2 * k], acc[o][2 * k + 1]));
                            }
                        }
                    }
                }
            }
        }
    }
    uint32_t *q = a.out + (size_t)i * COUT * 3;
#pragma unroll
    for (int o = 0; o < COUT; o++)
#pragma unroll
        for (int k = 0; k < 3; k++) q[o * 3 + k] = bf_pack(acc[o][2 * k], acc[o][2 * k + 1]);
}

// ---------------------------------------------------------------- 8 -> 8 layer on the tensor cores
// The channel mixing of a C -> C layer is a dense contraction: for each colour a,
//   y[x][a][c'] = sum_tap sum_c w[tap][c'][c] (T_tap psi_c)(x)[a],
// i.e. per tap a [sites x C] x [C x C] complex product, in real form
//   [Re y, Im y] = [Re t, Im t] [[Re w, Im w], [-Im w, Re w]]  (K = N = 2C = 16).
// A CTA takes 128 sites (one thread each, the MMA's M = 128 rows).  For every tap the
// threads gather and transport their 8 input channels on the CUDA cores, round them to
// BF16 and write one row per colour into a shared-memory A tile (no-swizzle K-major
// layout); one thread then issues three tcgen05.mma (one per colour, M = 128, N = 16,
// K = 16) that accumulate in FP32 in tensor memory, and commits them to the tap's
// mbarrier.  The A tiles form a two-stage ring: the transports of tap t + 1 overlap the
// MMAs of tap t.  The B tiles (17 taps of 16 x 16 BF16 weights in real form) are built
// once per CTA.  After the last tap the accumulators are read back with tcgen05.ld.
// Waits are bounded: a wait that runs out raises the context's device error flag and the
// layer's output is not written.
constexpr int kTcRows = 128;
constexpr int kTcCols = 64;                  // TMEM columns: 3 colours x N = 16 (power of two)
constexpr uint32_t kTcTile = 128 * 16 * 2;   // one A tile: 128 rows x 16 BF16
constexpr uint32_t kTcLBO = 128, kTcSBO = 256;

struct NetTcSmem {
    alignas(1024) uint8_t A[2][3][kTcTile];  // two stages x three colours
    alignas(128) uint8_t B[kNetTaps][512];   // per tap: 16 x 16 BF16, K-major
    uint64_t bar[2];
    uint64_t probe;                          // completed by nothing (self-test of the wait path)
    uint32_t tmem;
};

__device__ __forceinline__ uint32_t tc_off(uint32_t row, uint32_t k)
{
    return (row >> 3) * kTcSBO + (k >> 3) * kTcLBO + (row & 7) * 16 + (k & 7) * 2;
}

// raw loads of one tap of one site (issued one tap ahead of their use)
template <int PL>
struct TapLoad {
    static constexpr int LB = LinkBytes<PL>::b18;
    uint32_t lw[LB / 4];             // link words (taps 1..16)
    uint32_t act[kNetMaxChan * 3];   // the 8 input channels at the source site
};

template <int PL>
__device__ __forceinline__ void tap_issue(const NetLayerArgs &a, const Site &c, uint32_t s, int p, uint32_t i, int tap,
                                          TapLoad<PL> &L)
{
    uint32_t n = i;
    if (tap > 0) {
        const int k = tap - 1, type = k >= 8, mu = (k & 7) >> 1, back = k & 1;
        bool wrap;
        const uint32_t sn = neighbour(a.g, c, s, mu, type ? (back ? -3 : 3) : (back ? -1 : 1), wrap);
        const int lp = back ? 1 - p : p;
        const char *slot = a.links + (size_t)((lp * 2 + type) * 4 + mu) * a.slot_bytes;
        load_link_words<TapLoad<PL>::LB>(slot, back ? sn : s, L.lw);
        n = sn + (uint32_t)(1 - p) * a.g.Vh;
    }
    const uint4 *src = reinterpret_cast<const uint4 *>(a.in + (size_t)n * kNetMaxChan * 3);
#pragma unroll
    for (int q = 0; q < kNetMaxChan * 3 / 4; q++) {
        const uint4 v = __ldg(src + q);
        L.act[4 * q] = v.x;
        L.act[4 * q + 1] = v.y;
        L.act[4 * q + 2] = v.z;
        L.act[4 * q + 3] = v.w;
    }
}

// Persistent CTAs: each CTA allocates its TMEM columns, builds the B tiles and initialises
// its barriers once, then loops over tiles of 128 sites.  Per tap, the loads of the next
// tap are issued after the current tap's rows are written, so their latency overlaps the
// barrier and the MMA issue.
template <int PL>
__global__ void __launch_bounds__(128, 5) k_net_layer_tc(const NetLayerArgs a, DevStatus *status)
{
    constexpr int C = kNetMaxChan;
    __shared__ NetTcSmem sm;
    const int r = threadIdx.x, warp = r >> 5;
    // B tiles from the complex weights w[tap][c'][c]: rows n = 2c' + (0 re, 1 im), k = 2c + (0 re, 1 im)
    for (int q = r; q < kNetTaps * C * C; q += blockDim.x) {
        const int tap = q / (C * C), o = (q / C) % C, ci = q % C;
        // the links' per-type storage scale is folded into the weights of their taps
        const float ls = tap == 0 ? 1.f : a.scale[tap >= 9 ? 1 : 0];
        const float2 w = make_float2(a.w[q].x * ls, a.w[q].y * ls);
        uint8_t *bt = sm.B[tap];
        *reinterpret_cast<__nv_bfloat16 *>(bt + tc_off(2 * o, 2 * ci)) = __float2bfloat16_rn(w.x);
        *reinterpret_cast<__nv_bfloat16 *>(bt + tc_off(2 * o, 2 * ci + 1)) = __float2bfloat16_rn(-w.y);
        *reinterpret_cast<__nv_bfloat16 *>(bt + tc_off(2 * o + 1, 2 * ci)) = __float2bfloat16_rn(w.y);
        *reinterpret_cast<__nv_bfloat16 *>(bt + tc_off(2 * o + 1, 2 * ci + 1)) = __float2bfloat16_rn(w.x);
    }
    if (warp == 0) tc::tmem_alloc(&sm.tmem, kTcCols);
    if (r == 0) {
        tc::mbar_init(&sm.bar[0], 1);
        tc::mbar_init(&sm.bar[1], 1);
        tc::mbar_init(&sm.probe, 1);
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sm.tmem;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcRows, 2 * C);
    bool ok = true;
    // self-test: a bounded wait that runs out (nothing arrives on the probe barrier)
    if (a.selftest_wait) ok &= tc::mbar_wait(&sm.probe, 0, 1000000ull);

    // tiles alternate between the parities over the same half-sites (links reused in L2)
    const uint32_t tpp = (a.g.Vh + kTcRows - 1) / kTcRows; // tiles per parity
    const uint32_t ntiles = a.even_only_out ? tpp : 2 * tpp;
    uint32_t issued0 = 0u, issued1 = 0u; // commits on each stage so far (the same in every thread)
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int p = a.even_only_out ? 0 : (int)(tile & 1);
        const uint32_t s0 = (a.even_only_out ? tile : tile >> 1) * kTcRows + r;
        const bool live = s0 < a.g.Vh;
        const uint32_t s = live ? s0 : 0;
        const uint32_t i = s + (uint32_t)p * a.g.Vh;
        Site c{};
        if (live) c = site_coords(a.g, s, p);
        TapLoad<PL> L;
        if (live) tap_issue<PL>(a, c, s, p, i, 0, L);
        for (int tap = 0; tap < kNetTaps; tap++) {
            const int st = tap & 1;
            // the MMAs that last read this stage
            const uint32_t nst = st ? issued1 : issued0;
            if (nst > 0) ok &= tc::mbar_wait(&sm.bar[st], (nst - 1) & 1);
            uint32_t row[3][C]; // colour, channel: BF16 pair (re, im) of the transported input
            if (live) {
                if (tap > 0) {
                    // the stored link; its per-type scale is folded into the B tile
                    const int back = (tap - 1) & 1;
                    typename Prec<HISQ_F32>::Link U;
                    Prec<PL>::template unpack<18>(L.lw, U);
#pragma unroll
                    for (int ch = 0; ch < C; ch++) {
                        float v[6], t[6];
#pragma unroll
                        for (int k2 = 0; k2 < 3; k2++) {
                            v[2 * k2] = bf_lo(L.act[3 * ch + k2]);
                            v[2 * k2 + 1] = bf_hi(L.act[3 * ch + k2]);
                        }
                        transport(U, back, v, t);
#pragma unroll
                        for (int k2 = 0; k2 < 3; k2++) row[k2][ch] = bf_pack(t[2 * k2], t[2 * k2 + 1]);
                    }
                } else {
#pragma unroll
                    for (int ch = 0; ch < C; ch++)
#pragma unroll
                        for (int k2 = 0; k2 < 3; k2++) row[k2][ch] = L.act[3 * ch + k2];
                }
            } else {
#pragma unroll
                for (int k2 = 0; k2 < 3; k2++)
#pragma unroll
                    for (int ch = 0; ch < C; ch++) row[k2][ch] = 0u;
            }
#pragma unroll
            for (int k2 = 0; k2 < 3; k2++) {
                uint8_t *dst = sm.A[st][k2] + tc_off((uint32_t)r, 0);
                *reinterpret_cast<uint4 *>(dst) = make_uint4(row[k2][0], row[k2][1], row[k2][2], row[k2][3]);
                *reinterpret_cast<uint4 *>(dst + kTcLBO) = make_uint4(row[k2][4], row[k2][5], row[k2][6], row[k2][7]);
            }
            if (live && tap + 1 < kNetTaps) tap_issue<PL>(a, c, s, p, i, tap + 1, L);
            tc::fence_smem_to_async();
            __syncthreads();
            if (r == 0) {
                tc::fence_after_sync();
                const uint64_t bd = tc::sdesc(tc::smem_u32(sm.B[tap]), kTcLBO, kTcSBO);
#pragma unroll
                for (int k2 = 0; k2 < 3; k2++)
                    tc::mma_bf16(tmem + 2 * C * k2, tc::sdesc(tc::smem_u32(sm.A[st][k2]), kTcLBO, kTcSBO), bd, idesc,
                                 tap > 0);
                tc::commit(&sm.bar[st]);
            }
            if (st) issued1++;
            else issued0++;
        }
        // the last commit covers every MMA of the tile
        constexpr int last = (kNetTaps - 1) & 1;
        ok &= tc::mbar_wait(&sm.bar[last], ((last ? issued1 : issued0) - 1) & 1);
        tc::fence_after_sync();
        float d[3][2 * C];
#pragma unroll
        for (int k2 = 0; k2 < 3; k2++) tc::ld_32x32b_x16(tmem + ((uint32_t)(32 * warp) << 16) + 2 * C * k2, d[k2]);
        if (live && ok) {
            uint4 *q = reinterpret_cast<uint4 *>(a.out + (size_t)i * C * 3);
            uint32_t o[C * 3];
#pragma unroll
            for (int ch = 0; ch < C; ch++)
#pragma unroll
                for (int k2 = 0; k2 < 3; k2++) o[3 * ch + k2] = bf_pack(d[k2][2 * ch], d[k2][2 * ch + 1]);
#pragma unroll
            for (int j = 0; j < C * 3 / 4; j++) q[j] = make_uint4(o[4 * j], o[4 * j + 1], o[4 * j + 2], o[4 * j + 3]);
        }
        // the accumulator reads come before the next tile's first MMA (ordered by its barrier)
        tc::fence_before_sync();
    }
    if (!ok && status) {
        status->where = 1; // network tensor-core layer
        atomicExch(&status->error, (int)HISQ_EDEVICE);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTcCols);
}

// weight gradient: per block partial sums of G[tap][c'][c] (complex) -> part[block][17*cout*cin]
template <int PL, int CIN, int COUT>
__global__ void __launch_bounds__(128) k_net_wgrad(const NetLayerArgs a, const uint32_t *gout, float2 *part)
{
    __shared__ float2 sg[kNetTaps * COUT * CIN];
    for (int q = threadIdx.x; q < kNetTaps * COUT * CIN; q += blockDim.x) sg[q] = make_float2(0.f, 0.f);
    __syncthreads();
    const uint32_t V = 2 * a.g.Vh;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < V;
    const int p = live ? (i >= a.g.Vh) : 0;
    const uint32_t s = live ? i - p * a.g.Vh : 0;
    const int lane = threadIdx.x & 31;
    float g[COUT][6];
#pragma unroll
    for (int o = 0; o < COUT; o++) {
        if (live) load_chan<COUT>(gout, i, o, g[o]);
        else
#pragma unroll
            for (int k = 0; k < 6; k++) g[o][k] = 0.f;
    }
    const Site c = site_coords(a.g, s, p);
    for (int tap = 0; tap < kNetTaps; tap++) {
        typename Prec<HISQ_F32>::Link U;
        uint32_t n = i;
        bool back = false, zero = !live;
        if (tap > 0) {
            const int k = tap - 1, three = k >= 8, mu = (k & 7) >> 1, bk = k & 1;
            const int h = three * 2 + bk;
            uint32_t sn = 0;
            int type;
            if (live) {
                tap_link<PL>(a, c, s, p, mu, h, U, sn, back, type);
                n = sn + (uint32_t)(1 - p) * a.g.Vh;
            }
            if (a.even_only_in && p == 0) zero = true; // neighbours of even sites are odd
        } else if (a.even_only_in && p == 1) {
            zero = true;
        }
        for (int ci = 0; ci < CIN; ci++) {
            float t[6];
            if (!zero) {
                float v[6];
                load_chan<CIN>(a.in, n, ci, v);
                if (tap > 0) transport(U, back, v, t);
                else
#pragma unroll
                    for (int k = 0; k < 6; k++) t[k] = v[k];
            } else {
#pragma unroll
                for (int k = 0; k < 6; k++) t[k] = 0.f;
            }
#pragma unroll
            for (int o = 0; o < COUT; o++) {
                // conj(t) . g
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    re = fmaf(t[2 * k], g[o][2 * k], fmaf(t[2 * k + 1], g[o][2 * k + 1], re));
                    im = fmaf(t[2 * k], g[o][2 * k + 1], fmaf(-t[2 * k + 1], g[o][2 * k], im));
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    re += __shfl_xor_sync(0xffffffffu, re, off);
                    im += __shfl_xor_sync(0xffffffffu, im, off);
                }
                if (lane == 0) {
                    atomicAdd(&sg[(tap * COUT + o) * CIN + ci].x, re);
                    atomicAdd(&sg[(tap * COUT + o) * CIN + ci].y, im);
                }
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kNetTaps * COUT * CIN; q += blockDim.x)
        part[(size_t)blockIdx.x * kNetTaps * COUT * CIN + q] = sg[q];
}

// sum the block partials in a fixed order (FP64) and add to grad
__global__ void k_net_wgrad_reduce(const float2 *part, int nblocks, int nw, double2 *grad)
{
    const int q = blockIdx.x;
    double re = 0.0, im = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const float2 v = part[(size_t)b * nw + q];
        re += v.x;
        im += v.y;
    }
    re = block_sum(re);
    __syncthreads();
    im = block_sum(im);
    if (threadIdx.x == 0) {
        grad[q].x += re;
        grad[q].y += im;
    }
}

// w'[tap'][c][c'] = conj(w[adj(tap')][c'][c]) for the backward-data pass
__global__ void k_net_adjoint_weights(const float2 *w, float2 *wa, int cin, int cout)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNetTaps * cin * cout) return;
    const int tp = q / (cin * cout), rem = q % (cin * cout);
    const int ci = rem / cout, co = rem % cout; // wa layout [tap'][cin (now out)][cout (now in)]
    const int tap = tp == 0 ? 0 : (((tp - 1) ^ 1) + 1);
    const float2 v = w[(tap * cout + co) * cin + ci];
    wa[(tp * cin + ci) * cout + co] = make_float2(v.x, -v.y);
}

// b (canonical F64, even sites) -> 1-channel BF16 activation on the full lattice
__global__ void k_net_input(const double *b, uint32_t *act, uint32_t Vh)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * Vh) return;
#pragma unroll
    for (int k = 0; k < 3; k++)
        act[(size_t)i * 3 + k] = i < Vh ? bf_pack((float)b[(size_t)i * 6 + 2 * k], (float)b[(size_t)i * 6 + 2 * k + 1]) : 0u;
}

// z (canonical F64, even sites) from the 1-channel output activation
__global__ void k_net_output(const uint32_t *act, double *z, uint32_t Vh)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Vh) return;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const uint32_t w = act[(size_t)i * 3 + k];
        z[(size_t)i * 6 + 2 * k] = bf_lo(w);
        z[(size_t)i * 6 + 2 * k + 1] = bf_hi(w);
    }
}

// loss pieces: d = z - x on even sites; partial |d|^2 and |x|^2 (FIN_STORE values 0, 1)
__global__ void k_net_loss(const uint32_t *zact, const double *x, uint32_t Vh, Reduce red)
{
    double dd = 0.0, xx = 0.0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const uint32_t w = zact[(size_t)i * 3 + k];
            const double xr = x[(size_t)i * 6 + 2 * k], xi = x[(size_t)i * 6 + 2 * k + 1];
            const double dr = bf_lo(w) - xr, di = bf_hi(w) - xi;
            dd += dr * dr + di * di;
            xx += xr * xr + xi * xi;
        }
    }
    double mine[2] = {block_sum(dd), 0.0};
    __syncthreads();
    mine[1] = block_sum(xx);
    grid_reduce<2>(red, mine, 2, 0, 2, blockIdx.x);
}

// g = 2 (z - x) / |x|^2 on even sites, 0 on odd sites (1-channel BF16)
__global__ void k_net_loss_grad(const uint32_t *zact, const double *x, uint32_t *g, uint32_t Vh, const Scalars *sc,
                                double weight)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * Vh) return;
    const double f = weight * 2.0 / sc[1].last;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        uint32_t out = 0u;
        if (i < Vh) {
            const uint32_t w = zact[(size_t)i * 3 + k];
            out = bf_pack((float)(f * (bf_lo(w) - x[(size_t)i * 6 + 2 * k])),
                          (float)(f * (bf_hi(w) - x[(size_t)i * 6 + 2 * k + 1])));
        }
        g[(size_t)i * 3 + k] = out;
    }
}

// residual-loss pieces: |A e|^2 and |b|^2 (FIN_STORE values 0, 1)
__global__ void k_net_loss_res(const double *Ae, const double *b, uint32_t Vh, Reduce red)
{
    double rr = 0.0, bb = 0.0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const double a = Ae[(size_t)i * 6 + k], c = b[(size_t)i * 6 + k];
            rr += a * a;
            bb += c * c;
        }
    }
    double mine[2] = {rr, bb};
    block_sum_multi<2>(mine);
    grid_reduce<2>(red, mine, 2, 0, 2, blockIdx.x);
}

// e = z - x (canonical FP64)
__global__ void k_net_sub(const double *z, const double *x, double *e, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) e[i] = z[i] - x[i];
}

// g = weight * 2 A^2 e / |b|^2 on even sites, 0 on odd sites (1-channel BF16)
__global__ void k_net_grad_res(const double *A2e, uint32_t *g, uint32_t Vh, const Scalars *sc, double weight)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * Vh) return;
    const double f = weight * 2.0 / sc[1].last;
#pragma unroll
    for (int k = 0; k < 3; k++)
        g[(size_t)i * 3 + k] = i < Vh ? bf_pack((float)(f * A2e[(size_t)i * 6 + 2 * k]),
                                                (float)(f * A2e[(size_t)i * 6 + 2 * k + 1]))
                                      : 0u;
}

// ---------------------------------------------------------------- launch helpers
template <int PL>
static cudaError_t launch_layer_pl(const NetLayerArgs &a, int cin, int cout, cudaStream_t st)
{
    const unsigned nbp = (a.g.Vh + 127) / 128, nb = a.even_only_out ? nbp : 2 * nbp;
    if (cin == kNetMaxChan && cout == kNetMaxChan && a.tensor_cores && !a.even_only_in) {
        // persistent CTAs: at most the resident count (and at most 8 per SM, so that the
        // CTAs of one SM never ask for more than the 512 TMEM columns)
        // (resident CTAs per SM from the kernel's registers and shared memory, at most 8 so
        // that the CTAs of one SM never ask for more than the 512 TMEM columns)
        static int per_sm = -1, sms = 0;
        if (per_sm < 0) {
            int dev = 0, regs_sm = 0, smem_sm = 0, thr_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
            // the largest shared-memory carve-out, so that the register-limited count fits
            cudaFuncSetAttribute(k_net_layer_tc<PL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
            cudaFuncAttributes fa{};
            if (cudaFuncGetAttributes(&fa, k_net_layer_tc<PL>) == cudaSuccess && fa.numRegs > 0) {
                const int regs_cta = ((fa.numRegs + 7) / 8 * 8) * kTcRows;
                const int smem_cta = (int)fa.sharedSizeBytes + 1024; // + the per-CTA reservation
                per_sm = std::min({regs_sm / regs_cta, smem_sm / smem_cta, thr_sm / kTcRows, 512 / kTcCols});
            } else {
                per_sm = 0; // unknown: one CTA per tile
            }
            cudaGetLastError();
        }
        const unsigned tiles = nb;
        const unsigned grid = per_sm > 0 ? std::min<unsigned>(tiles, (unsigned)(per_sm * std::max(1, sms))) : tiles;
        k_net_layer_tc<PL><<<grid, kTcRows, 0, st>>>(a, a.status);
        return cudaGetLastError();
    }
#define HISQ_NET_CASE(CI, CO)                                                     \
    if (cin == CI && cout == CO) {                                                \
        k_net_layer<PL, CI, CO><<<nb, 128, 0, st>>>(a);                           \
        return cudaGetLastError();                                                \
    }
    HISQ_NET_CASE(1, kNetMaxChan) HISQ_NET_CASE(kNetMaxChan, kNetMaxChan) HISQ_NET_CASE(kNetMaxChan, 1)
    HISQ_NET_CASE(1, 1) HISQ_NET_CASE(1, 2) HISQ_NET_CASE(2, 2) HISQ_NET_CASE(2, 1) HISQ_NET_CASE(1, 4)
    HISQ_NET_CASE(4, 4) HISQ_NET_CASE(4, 1)
#undef HISQ_NET_CASE
    return cudaErrorInvalidValue;
}

template <int PL>
static cudaError_t launch_wgrad_pl(const NetLayerArgs &a, const uint32_t *g, float2 *part, int cin, int cout,
                                   cudaStream_t st)
{
    const unsigned V = 2 * a.g.Vh, nb = (V + 127) / 128;
#define HISQ_NET_CASE(CI, CO)                                                     \
    if (cin == CI && cout == CO) {                                                \
        k_net_wgrad<PL, CI, CO><<<nb, 128, 0, st>>>(a, g, part);                  \
        return cudaGetLastError();                                                \
    }
    HISQ_NET_CASE(1, kNetMaxChan) HISQ_NET_CASE(kNetMaxChan, kNetMaxChan) HISQ_NET_CASE(kNetMaxChan, 1)
    HISQ_NET_CASE(1, 1) HISQ_NET_CASE(1, 2) HISQ_NET_CASE(2, 2) HISQ_NET_CASE(2, 1) HISQ_NET_CASE(1, 4)
    HISQ_NET_CASE(4, 4) HISQ_NET_CASE(4, 1)
#undef HISQ_NET_CASE
    return cudaErrorInvalidValue;
}

bool net_shape_supported(int cin, int cout)
{
    const int ok[][2] = {{1, kNetMaxChan}, {kNetMaxChan, kNetMaxChan}, {kNetMaxChan, 1}, {1, 1}, {1, 2},
                         {2, 2}, {2, 1}, {1, 4}, {4, 4}, {4, 1}};
    for (auto &q : ok)
        if (q[0] == cin && q[1] == cout) return true;
    return false;
}

static NetLayerArgs layer_args(const hisq_net *n, const float2 *w, const uint32_t *in, uint32_t *out, int even_in,
                               int even_out = 0)
{
    NetLayerArgs a{};
    const LinkStore &L = n->ctx->links[n->link_prec];
    a.g = n->ctx->g;
    a.links = L.base;
    a.slot_bytes = L.slot_bytes;
    a.scale[0] = (float)L.scale[0];
    a.scale[1] = (float)L.scale[1];
    a.w = w;
    a.in = in;
    a.out = out;
    a.even_only_in = even_in;
    a.even_only_out = even_out;
    a.tensor_cores = n->opts.tensor_cores;
    a.selftest_wait = n->opts.selftest_wait;
    a.status = n->ctx->status;
    return a;
}

cudaError_t net_layer(const hisq_net *n, const float2 *w, const uint32_t *in, uint32_t *out, int cin, int cout,
                      int even_in, cudaStream_t st, int even_out = 0)
{
    const NetLayerArgs a = layer_args(n, w, in, out, even_in, even_out);
    return n->link_prec == HISQ_F16 ? launch_layer_pl<HISQ_F16>(a, cin, cout, st)
                                    : launch_layer_pl<HISQ_F32>(a, cin, cout, st);
}

cudaError_t net_wgrad(const hisq_net *n, const uint32_t *in, const uint32_t *g, float2 *part, int cin, int cout,
                      int even_in, cudaStream_t st)
{
    const NetLayerArgs a = layer_args(n, nullptr, in, nullptr, even_in);
    return n->link_prec == HISQ_F16 ? launch_wgrad_pl<HISQ_F16>(a, g, part, cin, cout, st)
                                    : launch_wgrad_pl<HISQ_F32>(a, g, part, cin, cout, st);
}

// z = K(b): b, z canonical complex128 [Vh][3] device buffers
int net_forward(hisq_net *n, const double *b, double *z, cudaStream_t st)
{
    const uint32_t Vh = n->ctx->g.Vh, V = 2 * Vh;
    k_net_input<<<(V + 255) / 256, 256, 0, st>>>(b, n->act[0], Vh);
    for (int l = 0; l < n->nlayer; l++) {
        // the output of the last layer is read on the even sites only
        cudaError_t e = net_layer(n, n->w + n->woff[l], n->act[l], n->act[l + 1], n->chans[l], n->chans[l + 1],
                                  l == 0, st, l == n->nlayer - 1);
        if (e != cudaSuccess) return cuda_error(n->ctx, e, "network layer");
    }
    if (z) k_net_output<<<(Vh + 255) / 256, 256, 0, st>>>(n->act[n->nlayer], z, Vh);
    HISQ_CUDA(n->ctx, cudaGetLastError());
    return HISQ_OK;
}

// one (b, x) pair: forward, loss, gradient accumulated into n->grad (weight `scale`)
int net_accumulate(hisq_net *n, const double *b, const double *x, double scale, cudaStream_t st)
{
    hisq_ctx *ctx = n->ctx;
    const uint32_t Vh = ctx->g.Vh, V = 2 * Vh;
    const bool res = n->opts.loss == 1;
    int rc = net_forward(n, b, res ? n->zb : nullptr, st);
    if (rc) return rc;
    Reduce R;
    R.partials = n->partials;
    R.counter = n->counter;
    R.sc = n->sc;
    R.op = FIN_STORE;
    R.nblocks = n->nblk_vec;
    R.ntotal = n->nblk_vec;
    if (res) { // e = K b - x; loss |A e|^2 / |b|^2; output gradient 2 A^2 e / |b|^2
        const size_t nd = (size_t)Vh * 6;
        k_net_sub<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(n->zb, x, n->eb, nd);
        const size_t rb = (size_t)Vh * 48;
        const double m = n->opts.mass;
        if ((rc = apply_mdagm(ctx, HISQ_F64, m, n->eb, n->tb, n->Aeb, 1, rb, st, nullptr, true))) return rc;
        if ((rc = apply_mdagm(ctx, HISQ_F64, m, n->Aeb, n->tb, n->A2eb, 1, rb, st, nullptr, true))) return rc;
        k_net_loss_res<<<n->nblk_vec, kVecBlock, 0, st>>>(n->Aeb, b, Vh, R);
        k_net_grad_res<<<(V + 255) / 256, 256, 0, st>>>(n->A2eb, n->gact[0], Vh, n->sc, scale);
    } else {
        k_net_loss<<<n->nblk_vec, kVecBlock, 0, st>>>(n->act[n->nlayer], x, Vh, R);
        k_net_loss_grad<<<(V + 255) / 256, 256, 0, st>>>(n->act[n->nlayer], x, n->gact[0], Vh, n->sc, scale);
    }
    HISQ_CUDA(n->ctx, cudaGetLastError());
    uint32_t *g = n->gact[0], *gnext = n->gact[1];
    for (int l = n->nlayer - 1; l >= 0; l--) {
        const int cin = n->chans[l], cout = n->chans[l + 1];
        const int nblocks = (int)((V + 127) / 128);
        cudaError_t e = net_wgrad(n, n->act[l], g, n->part, cin, cout, l == 0, st);
        if (e != cudaSuccess) return cuda_error(n->ctx, e, "network weight gradient");
        const int nw = kNetTaps * cin * cout;
        k_net_wgrad_reduce<<<nw, 256, 0, st>>>(n->part, nblocks, nw, n->grad + n->woff[l]);
        if (l > 0) {
            k_net_adjoint_weights<<<(nw + 127) / 128, 128, 0, st>>>(n->w + n->woff[l], n->wadj, cin, cout);
            e = net_layer(n, n->wadj, g, gnext, cout, cin, 0, st);
            if (e != cudaSuccess) return cuda_error(n->ctx, e, "network backward layer");
            std::swap(g, gnext);
        }
    }
    HISQ_CUDA(n->ctx, cudaGetLastError());
    return HISQ_OK;
}

}  // namespace hisq
