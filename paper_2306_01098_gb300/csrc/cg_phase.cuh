// cg_phase.cuh -- one phase of the mixed-precision CG (Sec. 3.2 "Inverters") in a single
// persistent, cooperatively launched kernel.
//
// Between two reliable updates the sloppy iterations of a single right-hand side run inside
// one launch: one block per SM, block b owning the half-lattice sites [b c, (b + 1) c) with
// c = ceil(Vh / blocks) rounded up to whole 32-site link blocks, one thread per site.  The
// iteration is the single-reduction arrangement of CG (the same recurrences as the CUDA-graph
// loop with single_reduction = 1):
//   t  = D_oe p                                                    [grid barrier]
//   Ap = m4 p - D_eo t;  <p,Ap>, |r|^2, <r,Ap>, <Ap,Ap> per block    [grid barrier]
//   every block sums the block partials in the same fixed order, so all blocks hold the
//   same alpha = |r|^2/<p,Ap>, |r - alpha Ap|^2 = |r|^2 - 2 alpha <r,Ap> + alpha^2 <Ap,Ap>,
//   beta and stop decision (fin_ab, shared with the multi-kernel path)
//   x += alpha p;  r -= alpha Ap;  p = r + beta p                    [grid barrier]
// Three barriers per iteration replace the four kernel launches of the graph loop, whose
// launch gaps are a large part of an iteration on lattices that fill about one wave.
// Only p (gathered by D_oe at the neighbours) and t (gathered by D_eo) travel through global
// memory; x, r, Ap and the block's own copy of p are read and written only at the block's own
// sites, so they stay in shared memory for the whole launch (loaded at entry, x and r written
// back at exit).  p and t are read with ordinary (coherent) loads, links with the read-only
// path.  The barrier has no shared counter: each block publishes its arrival (and, after the
// normal operator, its four partial sums) in its own 64-byte record, and every block polls all
// records.  Each wait is bounded (globaltimer): a wait that runs out raises the context's
// device error flag and ends the launch early; the host turns the flag into HISQ_EDEVICE.
#pragma once

#include <cstddef>

#include "blas.cuh"
#include "dslash_kernel.cuh"

namespace hisq {

// Launch shapes (threads per block NT, prefetch PF), chosen by code:
//   1: NT 1024     2: NT 512, PF     3: NT 896, PF     4: NT 1024, PF     5: NT 448, PF
// PF issues the loads of all four hops of a direction before their products; fewer threads
// per block leave it the registers that needs (a block of NT threads walks its c sites in
// ceil(c / NT) passes).

// Arrival record of one block (one 64-byte line): the number of grid barriers it has passed
// and, at the barrier after the normal operator, its partial sums of the four dot products
// (float-float pairs).
struct PhaseSlot {
    FF part[4]; // first: 16-byte aligned for the paired loads that copy it
    unsigned gen;
    unsigned pad;
    double pad2[3];
};
static_assert(sizeof(PhaseSlot) == 64, "one arrival record per 64-byte line");
static_assert(offsetof(PhaseSlot, part) % 16 == 0, "partial sums are read as 16-byte pairs");
constexpr int kPhaseMaxBlocks = 1024;
// shared memory per owned site: x, r, p, Ap (FP32 records)
constexpr int kPhaseSmemPerSite = 4 * 24;
constexpr int kPhaseMaxSmem = 200 * 1024;

struct PhaseArgs {
    DslashArgs doe;       // t = D_oe p   (output parity 1; in = p, out = t)
    DslashArgs deo;       // Ap = m4 p - D_eo t (output parity 0; in = t, m4)
    char *x, *p, *r;      // FP32 iteration vectors (24-byte records) in global memory
    uint32_t Vh;
    uint32_t chunk;       // sites per block (multiple of 32)
    Scalars *sc;          // scalars of the right-hand side: read at entry, written at exit
    PhaseSlot *slots;     // one per block, zeroed before the launch
    DevStatus *status;    // device error flag
    int cap;              // iterations this launch may run
    int it_end;           // and no iteration once Scalars.it_all reaches this (the solve's budget)
    unsigned long long wait_ns; // bound on one barrier wait
    int selftest;         // block 0 ends at once without arriving: the others' first wait runs out
    int reortho;          // the launch follows a reliable update: re-orthogonalise p against r first
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long phase_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier number g of a cooperative launch (every block resident).  After the
// block's threads meet, thread 0 writes the block's partial sums (if any) and releases g in
// the block's own record; the release orders every write the block made before the meeting.
// Thread i < gridDim.x of every block then waits until record i shows g (relaxed polling,
// then one acquire fence by the same thread), at most limit_ns.  Returns false, with the
// device error flag raised, if a wait ran out.
// With spart (shared memory, [4][gridDim.x]), the thread that waited for record i also copies
// that block's partial sums there, so all of them arrive in one parallel round trip.
__device__ __forceinline__ bool grid_barrier(PhaseSlot *slots, unsigned g, const FF *mine, DevStatus *st,
                                            unsigned long long limit_ns, FF *spart = nullptr)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        if (mine)
            for (int j = 0; j < 4; j++) slots[blockIdx.x].part[j] = mine[j];
        st_release_gpu(&slots[blockIdx.x].gen, g);
    }
    int good = 1;
    if (threadIdx.x < gridDim.x) {
        const unsigned *f = &slots[threadIdx.x].gen;
        unsigned long long t0 = 0;
        int n = 0;
        while ((int)(ld_relaxed_gpu(f) - g) < 0) {
            if (++n < 128) continue;
            n = 0;
            const unsigned long long t = phase_clock_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) {
                good = 0;
                break;
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (spart && good) {
            const float4 *q = reinterpret_cast<const float4 *>(slots[threadIdx.x].part);
            const float4 a0 = __ldcg(q), a1 = __ldcg(q + 1);
            spart[threadIdx.x] = FF{a0.x, a0.y};
            spart[gridDim.x + threadIdx.x] = FF{a0.z, a0.w};
            spart[2 * gridDim.x + threadIdx.x] = FF{a1.x, a1.y};
            spart[3 * gridDim.x + threadIdx.x] = FF{a1.z, a1.w};
        }
    }
    good = __syncthreads_and(good);
    if (!good && threadIdx.x == 0) {
        atomicExch(&st->where, 2);
        atomicExch(&st->error, (int)HISQ_EDEVICE);
    }
    return good != 0;
}

// The same totals in every block: warp j < NV sums value j of the G block partials (copied
// to shared memory by the barrier), lane i taking blocks i, i + 32, ..., then a fixed tree;
// float-float throughout, one FP64 conversion per value.  Valid after the call's barrier.
template <int NV>
__device__ __forceinline__ void phase_totals(const FF *spart, uint32_t G, double *tot)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w < NV) {
        FF acc = {0.f, 0.f};
        for (uint32_t i = l; i < G; i += 32) ff_merge(acc, spart[w * G + i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const FF y = {__shfl_down_sync(0xffffffffu, acc.h, o), __shfl_down_sync(0xffffffffu, acc.l, o)};
            ff_merge(acc, y);
        }
        if (l == 0) tot[w] = ff_value(acc);
    }
    __syncthreads();
}

// PL: sloppy link storage (F32, F16, BF16) with NREAL reals; vectors FP32; NT threads per
// block; PF prefetch of a direction's four hops.  Dynamic shared memory: x, r, p, Ap of the
// block's sites (a.chunk records of 24 bytes each), then [4][gridDim.x] partial sums.
template <int PL, int NREAL, int NT, bool PF>
__global__ void __launch_bounds__(NT, 1) k_cg_phase(const PhaseArgs a)
{
    using T = Prec<HISQ_F32>;
    using B = Blas<HISQ_F32>;
    extern __shared__ __align__(16) char phase_smem[];
    __shared__ Scalars S;
    __shared__ double tot[4];
    __shared__ float coef[3];
    __shared__ int mode, xr_on;
    if (a.selftest && blockIdx.x == 0) return;
    const uint32_t cbeg = min(a.Vh, blockIdx.x * a.chunk), cend = min(a.Vh, cbeg + a.chunk);
    char *sx = phase_smem, *sr = sx + (size_t)a.chunk * 24, *sp = sr + (size_t)a.chunk * 24;
    char *sAp = sp + (size_t)a.chunk * 24;
    FF *spart = reinterpret_cast<FF *>(sAp + (size_t)a.chunk * 24); // [4][gridDim.x]
    for (uint32_t s = cbeg + threadIdx.x; s < cend; s += NT) {
        typename B::Vec v;
        T::load_coh(a.x, s, v);
        B::store(sx, s - cbeg, v);
        T::load_coh(a.r, s, v);
        B::store(sr, s - cbeg, v);
        T::load_coh(a.p, s, v);
        B::store(sp, s - cbeg, v);
    }
    if (threadIdx.x == 0) S = *a.sc;
    __syncthreads();
    const uint32_t G = gridDim.x;
    unsigned g = 0; // grid barriers passed
    bool ok = true;
    // After a reliable update replaced r: remove from p its component along r, then
    // p = r + beta p, i.e. p = (1 - beta <r,p>/|r|^2) r + beta p with the complex
    // <r,p> = sum conj(r) p over the lattice: per-site products in FP32, float-float sums in
    // the block, block partials through the barrier's records (summed in the same order by
    // every block), the coefficients in FP64 and the update in FP32 like the iterations'.
    if (a.reortho && S.active) {
        FF d[2] = {{0.f, 0.f}, {0.f, 0.f}};
        for (uint32_t s = cbeg + threadIdx.x; s < cend; s += NT) {
            typename B::Vec pv, rv;
            T::load_coh(sp, s - cbeg, pv);
            T::load_coh(sr, s - cbeg, rv);
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                re = fmaf(rv.v[2 * i], pv.v[2 * i], fmaf(rv.v[2 * i + 1], pv.v[2 * i + 1], re));
                im = fmaf(rv.v[2 * i], pv.v[2 * i + 1], fmaf(-rv.v[2 * i + 1], pv.v[2 * i], im));
            }
            ff_add(d[0], re);
            ff_add(d[1], im);
        }
        block_sum_ff<2>(d);
        const FF mine[4] = {d[0], d[1], {0.f, 0.f}, {0.f, 0.f}};
        ok = grid_barrier(a.slots, ++g, mine, a.status, a.wait_ns, spart);
        if (ok) {
            phase_totals<2>(spart, G, tot);
            if (threadIdx.x == 0) {
                const double beta = S.beta, rr = S.rr;
                coef[0] = (float)(rr > 0.0 ? 1.0 - beta * tot[0] / rr : 1.0);
                coef[1] = (float)(rr > 0.0 ? -beta * tot[1] / rr : 0.0);
                coef[2] = (float)beta;
            }
            __syncthreads();
            const float cre = coef[0], cim = coef[1], bf = coef[2];
            for (uint32_t s = cbeg + threadIdx.x; s < cend; s += NT) {
                typename B::Vec pv, rv, out;
                T::load_coh(sp, s - cbeg, pv);
                T::load_coh(sr, s - cbeg, rv);
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const float xr = rv.v[2 * i], xi = rv.v[2 * i + 1], yr = pv.v[2 * i], yi = pv.v[2 * i + 1];
                    out.v[2 * i] = fmaf(cre, xr, fmaf(-cim, xi, bf * yr));
                    out.v[2 * i + 1] = fmaf(cre, xi, fmaf(cim, xr, bf * yi));
                }
                B::store(sp, s - cbeg, out);
                B::store(a.p, s, out);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                S.last = tot[0];
                S.last_im = tot[1];
            }
            // p complete everywhere before the first D_oe gathers it
            ok = grid_barrier(a.slots, ++g, nullptr, a.status, a.wait_ns);
        }
    }
    for (int it = 0; ok && it < a.cap && S.it_all < a.it_end && S.active; it++) {
        // t = D_oe p (p gathered from global memory)
        {
            FF none[1] = {{0.f, 0.f}};
            for (uint32_t s = cbeg + threadIdx.x; s < cend; s += NT)
                dslash_item<PL, HISQ_F32, NREAL, 1, 0, 1, true, PF, 1, FF>(
                    a.doe, a.doe.g, a.doe.links, a.doe.slot_bytes, a.doe.scale_f[0], a.doe.scale_f[1], a.doe.in,
                    a.doe.out, nullptr, nullptr, nullptr, 0u, none, s);
        }
        if (!(ok = grid_barrier(a.slots, ++g, nullptr, a.status, a.wait_ns))) break;
        // Ap = m4 p - D_eo t into shared memory, with the four dot products of the
        // single-reduction step (per-site products in FP32, float-float sums in the block);
        // the block sums travel with the barrier's arrival record
        {
            FF d[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            for (uint32_t s = cbeg + threadIdx.x; s < cend; s += NT)
                dslash_item<PL, HISQ_F32, NREAL, 1, 2, 1, true, PF, 1, FF>(
                    a.deo, a.deo.g, a.deo.links, a.deo.slot_bytes, a.deo.scale_f[0], a.deo.scale_f[1], a.deo.in, sAp,
                    sp, sr, nullptr, 0u, d, s, cbeg);
            block_sum_ff<4>(d);
            if (!(ok = grid_barrier(a.slots, ++g, d, a.status, a.wait_ns, spart))) break;
        }
        phase_totals<4>(spart, G, tot);
        // the scalars (FP64, one thread), then their float images for the update
        if (threadIdx.x == 0) {
            S.pAp = tot[0];
            S.last_im = tot[1];
            S.last = tot[2];
            fin_ab(S, tot[3]);
            // last iteration of the launch: p is left to the re-orthogonalisation after the update
            mode = it + 1 >= a.cap || S.it_all >= a.it_end ? 1 : 0;
            const double alpha = alpha_fresh_for_x(S) ? S.alpha : 0.0;
            coef[0] = (float)alpha;
            coef[1] = (float)S.beta;
            xr_on = alpha != 0.0;
        }
        __syncthreads();
        // x += alpha p ; r -= alpha Ap ; p = r + beta p  (alpha only if this iteration made it),
        // in FP32 like the multi-kernel loop's updates; the new p also goes to global memory
        // for the next D_oe
        {
            const float af = coef[0], bf = coef[1];
            const bool do_xr = xr_on != 0;
            const bool do_p = mode == 0 && S.active;
            for (uint32_t s = cbeg + threadIdx.x; s < cend; s += NT) {
                const uint32_t i = s - cbeg;
                typename B::Vec pv, rv;
                T::load_coh(sp, i, pv);
                T::load_coh(sr, i, rv);
                if (do_xr) {
                    typename B::Vec xv, av;
                    T::load_coh(sx, i, xv);
                    T::load_coh(sAp, i, av);
#pragma unroll
                    for (int k = 0; k < 6; k++) {
                        xv.v[k] = fmaf(af, pv.v[k], xv.v[k]);
                        rv.v[k] = fmaf(-af, av.v[k], rv.v[k]);
                    }
                    B::store(sx, i, xv);
                    B::store(sr, i, rv);
                }
                if (do_p) {
#pragma unroll
                    for (int k = 0; k < 6; k++) pv.v[k] = fmaf(bf, pv.v[k], rv.v[k]);
                    B::store(sp, i, pv);
                    B::store(a.p, s, pv);
                }
            }
        }
        // p complete everywhere before the next D_oe gathers it
        if (mode == 0 && S.active) ok = grid_barrier(a.slots, ++g, nullptr, a.status, a.wait_ns);
    }
    // x and r back to global memory (p is there already)
    __syncthreads();
    for (uint32_t s = cbeg + threadIdx.x; s < cend; s += NT) {
        typename B::Vec v;
        T::load_coh(sx, s - cbeg, v);
        B::store(a.x, s, v);
        T::load_coh(sr, s - cbeg, v);
        B::store(a.r, s, v);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && ok) *a.sc = S;
}

// sites per block for one block per SM (whole 32-site link blocks), 0 if the block's
// vectors would not fit in shared memory
inline uint32_t phase_chunk(uint32_t Vh, int sms)
{
    const uint32_t c = ((Vh + (uint32_t)sms - 1) / (uint32_t)sms + 31u) & ~31u;
    return (size_t)c * kPhaseSmemPerSite + 4 * sizeof(FF) * (size_t)sms <= (size_t)kPhaseMaxSmem ? c : 0u;
}

// one block per SM; every block polls every record, so blocks <= NT
template <int PL, int NREAL, int NT, bool PF>
static cudaError_t launch_phase_t(const PhaseArgs &a0, int sms, cudaStream_t st)
{
    PhaseArgs a = a0;
    a.chunk = phase_chunk(a.Vh, sms);
    if (a.chunk == 0 || sms > NT || sms > kPhaseMaxBlocks) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)a.chunk * kPhaseSmemPerSite + 4 * sizeof(FF) * (size_t)sms;
    // a per-device attribute of the function: set for the current device at every launch
    cudaError_t e0 = cudaFuncSetAttribute(k_cg_phase<PL, NREAL, NT, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kPhaseMaxSmem);
    if (e0 != cudaSuccess) return e0;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_phase<PL, NREAL, NT, PF>, NT, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)sms);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_cg_phase<PL, NREAL, NT, PF>, a);
}

template <int PL, int NREAL>
cudaError_t launch_phase_shape(const PhaseArgs &a, int shape, int sms, cudaStream_t st)
{
    switch (shape) {
    case 1: return launch_phase_t<PL, NREAL, 1024, false>(a, sms, st);
    case 2: return launch_phase_t<PL, NREAL, 512, true>(a, sms, st);
    case 3: return launch_phase_t<PL, NREAL, 896, true>(a, sms, st);
    case 4: return launch_phase_t<PL, NREAL, 1024, true>(a, sms, st);
    case 5: return launch_phase_t<PL, NREAL, 448, true>(a, sms, st);
    }
    return cudaErrorInvalidValue;
}

template <int PL>
cudaError_t launch_phase_pl(const PhaseArgs &a, int nreal, int shape, int sms, cudaStream_t st)
{
    return nreal == 12 ? launch_phase_shape<PL, 12>(a, shape, sms, st) : launch_phase_shape<PL, 18>(a, shape, sms, st);
}

#define HISQ_PHASE_INSTANTIATE(PL)                                                                      \
    cudaError_t phase_launch_##PL(const PhaseArgs &a, int nreal, int shape, int sms, cudaStream_t st)  \
    {                                                                                                  \
        return launch_phase_pl<PL>(a, nreal, shape, sms, st);                                          \
    }

}  // namespace hisq
