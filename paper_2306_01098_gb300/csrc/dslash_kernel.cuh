// dslash_kernel.cuh -- the HISQ staggered Dslash (Sec. 5.1) on one parity, all storage precisions.
//
//   out(x) = sum_mu [ X_mu(x) phi(x+mu) - X_mu(x-mu)^+ phi(x-mu)
//                   + W_mu(x) phi(x+3mu) - W_mu(x-3mu)^+ phi(x-3mu) ]      (x of parity p)
// with the staggered phases and the antiperiodic time boundary folded into the stored
// links (18 reals) or applied here (12 reals: rows 0 and 1 carry the sign, row 2 is
// rebuilt and signed in registers).
//
// Work decomposition
//   * NR right-hand sides per thread (the paper's N_inner loop, Sec. 5.1): every link is
//     loaded once per NR vectors.  The groups of NR right-hand sides (N_outer) are the
//     fastest index of the block number, so the blocks that read one tile of links run
//     together and only the first takes the links from HBM.
//   * Launch order of the sites: storage order, or with z and t interchanged (t runs
//     fastest among the planes).  A site's +-1/+-3 neighbours along the slowest launch
//     dimension were touched 1 to 3 slowest-dimension slices earlier; interchanging z and
//     t when Nt < Nz shrinks that reuse distance, and with it the L2 footprint that keeps
//     neighbour spinors of many right-hand sides resident.  Link stores too large for L2
//     are then read with an evict-first policy so that the streamed links do not displace
//     the spinors.
//   * DS threads per site (1, 2 or 4), each taking 4/DS of the directions; the partial sums
//     meet through warp shuffles.  On small lattices one thread per site leaves a single
//     short wave whose duration is the latency of 16 dependent gathers; splitting the
//     directions multiplies the loads in flight.
//   * Links (PL) stream through with L1-bypassing 16-byte loads, read once per application;
//     neighbour spinors (PV) are gathered through L1/L2, where their 16-fold reuse happens.
//     PL and PV differ only for 16-bit links with FP32 vectors.
// Optional epilogue (normal operator, Sec. 3.2 applyMdaggM):
//   EPI = 1: out = m4 * p - D in,   and <p, out> reduced in FP64 per right-hand side;
//   EPI = 2: the same and also |r|^2, <r, out> and <out, out> (four values per right-hand
//            side, from which the CG finishing step gets alpha and the next |r|^2).
// Batches: one launch over the lattices of a batch, each with its own geometry and links
// (one right-hand side per lattice); a block finds its lattice in the batch table.
#pragma once

#include <algorithm>

#include "arith.cuh"
#include "dslash.cuh"
#include "reduce.cuh"

namespace hisq {

// dot products per right-hand side reduced by an epilogue
template <int EPI> struct EpiDots { static constexpr int n = EPI == 2 ? 4 : 1; };

// |v|^2 and |o|^2 of FP32 records in float arithmetic, returned as floats
__device__ __forceinline__ float vec_norm2f(const FloatArith::Vec &v)
{
    float d = 0.f;
#pragma unroll
    for (int i = 0; i < 6; i++) d = fmaf(v.v[i], v.v[i], d);
    return d;
}
__device__ __forceinline__ float acc_norm2f(const FloatArith::Acc &o)
{
    float d = 0.f;
#pragma unroll
    for (int i = 0; i < 6; i++) d = fmaf(o.v[i], o.v[i], d);
    return d;
}

// |v|^2 of a vector: float arithmetic for the float types, double otherwise
template <class T>
__device__ __forceinline__ double vec_norm2(const typename T::Vec &v)
{
    if constexpr (std::is_same<typename T::Vec, FloatArith::Vec>::value) {
        float d = 0.f;
#pragma unroll
        for (int i = 0; i < 6; i++) d = fmaf(v.v[i], v.v[i], d);
        return (double)d;
    } else {
        double d = 0.0;
#pragma unroll
        for (int i = 0; i < 6; i++) {
            const double c = T::vcomp(v, i);
            d = fma(c, c, d);
        }
        return d;
    }
}

// |o|^2 of an accumulator: float arithmetic for the float types, double otherwise
template <class T>
__device__ __forceinline__ double acc_norm2(const typename T::Acc &o)
{
    if constexpr (std::is_same<typename T::Acc, FloatArith::Acc>::value) {
        float d = 0.f;
#pragma unroll
        for (int i = 0; i < 6; i++) d = fmaf(o.v[i], o.v[i], d);
        return (double)d;
    } else {
        double d = 0.0;
#pragma unroll
        for (int i = 0; i < 6; i++) {
            const double c = T::comp(o, i);
            d = fma(c, c, d);
        }
        return d;
    }
}

// vector load: the read-only path, or (COH) ordinary loads for vectors that other blocks of
// the same launch write between grid barriers
template <class T, bool COH>
__device__ __forceinline__ void vec_load(const char *base, uint32_t s, typename T::Vec &v)
{
    if constexpr (COH) T::load_coh(base, s, v);
    else T::load(base, s, v);
}

// One work item: the sites of one tile (a.bs threads, DS per site; this thread is
// number tid of the tile) for the NR right-hand sides whose vectors start at in/out/pv/rv
// (consecutive right-hand sides a.rhs_bytes apart); geometry g, link store `links`.
// Epilogue dot products are added to dots (value j of right-hand side r at
// dots[r * EpiDots<EPI>::n + j]).  With an epilogue, pv, rv and the output are addressed at
// site s - ebase (ebase = 0: the whole field; else a block's own range, e.g. in shared memory).
// PF: issue the loads of all four hops of a direction before their products (more requests
// in flight per thread, more registers).
// RG > 1 (with DS = 1): RG consecutive threads share a site, thread g of them taking the NR
// right-hand sides g NR .. g NR + NR - 1 from the given ones; their loads of the site's links
// are the same addresses in the same instruction (one request), so a link is fetched once
// for all NR RG right-hand sides with 1/RG of the accumulators per thread.
// LL1: links allocate in L1 (right-hand-side groups of one block read the same links).
template <int PL, int PV, int NREAL, int NR, int EPI, int DS, bool COH = false, bool PF = false, int RG = 1,
          class DT = double, bool LL1 = false>
__device__ __forceinline__ void dslash_item(const DslashArgs &a, const Geom &g, const char *links, size_t slot_bytes,
                                            std::conditional_t<std::is_same<DT, FF>::value, float, double> sc0,
                                            std::conditional_t<std::is_same<DT, FF>::value, float, double> sc1,
                                            const char *in, char *outp, const char *pvp,
                                            const char *rvp, const double *m4r, uint32_t tile,
                                            DT (&dots)[NR * EpiDots<EPI>::n], uint32_t tid = threadIdx.x,
                                            uint32_t ebase = 0)
{
    static_assert(RG == 1 || DS == 1, "right-hand side groups share a site only with one thread per direction set");
    constexpr int ND = EpiDots<EPI>::n;
    // DT = FF (FP32 vectors inside the persistent CG kernel): float-float dot sums, float
    // scales (sc0, sc1) and the float m4f, so that no FP64 conversion runs per site
    constexpr bool FFD = std::is_same<DT, FF>::value;
    static_assert(!FFD || std::is_same<typename Prec<PV>::Vec, FloatArith::Vec>::value,
                  "float-float dot sums are for FP32 iteration vectors");
    using T = Prec<PV>;  // vectors and arithmetic
    using TL = Prec<PL>; // link storage
    constexpr int LB = NREAL == 18 ? LinkBytes<PL>::b18 : LinkBytes<PL>::b12;
    constexpr bool TWO = (PL == HISQ_F16 || PL == HISQ_BF16 || NREAL == 12);
    constexpr bool SPLIT = T::kSplitDirections;
    constexpr int NMU = 4 / DS;
    const uint32_t gt = tile * (uint32_t)a.bs + tid;
    const uint32_t u = gt / (DS * RG); // site number in launch order
    const int part = (int)(gt % DS);
    if constexpr (RG > 1) {
        const size_t goff = (size_t)(gt % RG) * NR * a.rhs_bytes;
        in += goff;
        outp += goff;
        if (pvp) pvp += goff;
        if (rvp) rvp += goff;
        if (m4r) m4r += (gt % RG) * NR;
    }
    const bool live = u < g.Vh;
    uint32_t s = u;
    if (a.zt) { // u = ((z Nt + t) Ps + i)  ->  s = ((t Nz + z) Ps + i), Ps = sites of one plane
        const uint32_t plane = g.dp.div(u);
        const uint32_t z = g.dt.div(plane);
        s = ((plane - z * (uint32_t)g.n[3]) * (uint32_t)g.n[2] + z) * g.sz + (u - plane * g.sz);
    }
    typename T::Acc out[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) T::zero(out[r]);

    if (live) {
        const Site c = site_coords(g, s, a.p);
        typename T::Acc acc[TWO ? 2 : 1][NR];
#pragma unroll
        for (int t = 0; t < (TWO ? 2 : 1); t++)
#pragma unroll
            for (int r = 0; r < NR; r++) T::zero(acc[t][r]);

#pragma unroll
        for (int m = 0; m < NMU; m++) {
            const int mu = part * NMU + m;
            typename T::Acc dacc[SPLIT ? NR : 1];
            if constexpr (SPLIT) {
#pragma unroll
                for (int r = 0; r < NR; r++) T::zero(dacc[r]);
            }
            if constexpr (PF) {
                // the loads of all four hops first (8 to 12 independent requests per thread in
                // flight at once), then their products
                uint32_t w[4][LB / 4];
                typename T::Vec v[4][NR];
                bool wrap[4];
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    const int k = h == 0 ? 1 : h == 1 ? -1 : h == 2 ? 3 : -3;
                    const int type = h >> 1;
                    const bool back = h & 1;
                    const uint32_t sn = neighbour(g, c, s, mu, k, wrap[h]);
                    const int lp = back ? 1 - a.p : a.p;
                    const char *slot = links + (size_t)((lp * 2 + type) * 4 + mu) * slot_bytes;
                    load_link_words<LB, LL1>(slot, back ? sn : s, w[h], NR > 1 && a.stream_links != 0);
#pragma unroll
                    for (int r = 0; r < NR; r++) vec_load<T, COH>(in + (size_t)r * a.rhs_bytes, sn, v[h][r]);
                }
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    const int type = h >> 1;
                    const bool back = h & 1;
                    typename T::Link U;
                    TL::template unpack<NREAL>(w[h], U);
                    if constexpr (NREAL == 12) T::rebuild(U, (eta_neg(c, mu) != 0) ^ (mu == 3 && wrap[h]));
#pragma unroll
                    for (int r = 0; r < NR; r++) {
                        typename T::Acc &dst = SPLIT ? dacc[SPLIT ? r : 0] : acc[TWO ? type : 0][r];
                        if (back) T::template hop<true, true>(dst, U, v[h][r]);
                        else T::template hop<false, false>(dst, U, v[h][r]);
                    }
                }
            } else {
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const int k = h == 0 ? 1 : h == 1 ? -1 : h == 2 ? 3 : -3;
                const int type = h >> 1;
                const bool back = h & 1;
                bool wrap;
                const uint32_t sn = neighbour(g, c, s, mu, k, wrap);
                const int lp = back ? 1 - a.p : a.p;
                const char *slot = links + (size_t)((lp * 2 + type) * 4 + mu) * slot_bytes;
                uint32_t w[LB / 4];
                load_link_words<LB, LL1>(slot, back ? sn : s, w, NR > 1 && a.stream_links != 0);
                typename T::Link U;
                TL::template unpack<NREAL>(w, U);
                if constexpr (NREAL == 12) T::rebuild(U, (eta_neg(c, mu) != 0) ^ (mu == 3 && wrap));
#pragma unroll
                for (int r = 0; r < NR; r++) {
                    typename T::Vec v;
                    vec_load<T, COH>(in + (size_t)r * a.rhs_bytes, sn, v);
                    typename T::Acc &dst = SPLIT ? dacc[SPLIT ? r : 0] : acc[TWO ? type : 0][r];
                    if (back) T::template hop<true, true>(dst, U, v);
                    else T::template hop<false, false>(dst, U, v);
                }
            }
            }
            if constexpr (SPLIT) {
#pragma unroll
                for (int r = 0; r < NR; r++) {
                    if (m == 0) acc[0][r] = dacc[r];
                    else T::add_acc(acc[0][r], dacc[r]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < NR; r++) {
            if constexpr (TWO) {
                T::axpy_acc(out[r], (typename T::Real)sc0, acc[0][r]);
                T::axpy_acc(out[r], (typename T::Real)sc1, acc[1][r]);
            } else {
                out[r] = acc[0][r];
            }
        }
    }
    // partial sums of the DS threads of a site meet in every one of them
    if constexpr (DS > 1) {
#pragma unroll
        for (int off = DS / 2; off > 0; off >>= 1)
#pragma unroll
            for (int r = 0; r < NR; r++) T::shfl_xor_add(out[r], off);
    }
    if (live && part == 0) {
#pragma unroll
        for (int r = 0; r < NR; r++) {
            if constexpr (EPI >= 1) {
                typename T::Vec pv;
                vec_load<T, COH>(pvp + (size_t)r * a.rhs_bytes, s - ebase, pv);
                if constexpr (FFD) {
                    T::mdagm_epilogue(out[r], m4r ? a.m4f + (float)m4r[r] : a.m4f, pv);
                    ff_add(dots[r * ND], T::dotf(pv, out[r]));
                } else {
                    T::mdagm_epilogue(out[r], a.m4 + (m4r ? m4r[r] : 0.0), pv);
                    dots[r * ND] += T::dot(pv, out[r]);
                }
                if constexpr (EPI == 2) {
                    typename T::Vec rv;
                    vec_load<T, COH>(rvp + (size_t)r * a.rhs_bytes, s - ebase, rv);
                    if constexpr (FFD) {
                        ff_add(dots[r * ND + 1], vec_norm2f(rv));
                        ff_add(dots[r * ND + 2], T::dotf(rv, out[r]));
                        ff_add(dots[r * ND + 3], acc_norm2f(out[r]));
                    } else {
                        dots[r * ND + 1] += vec_norm2<T>(rv);
                        dots[r * ND + 2] += T::dot(rv, out[r]);
                        dots[r * ND + 3] += acc_norm2<T>(out[r]);
                    }
                }
            }
            T::store(outp + (size_t)r * a.rhs_bytes, EPI >= 1 ? s - ebase : s, out[r]);
        }
    }
}

// block sums of the epilogue's dot products (valid on thread 0): float-float or FP64
template <bool FFK, int N, class D>
__device__ __forceinline__ void block_sum_dots(D (&d)[N])
{
    if constexpr (FFK) block_sum_ff<N>(d);
    else block_sum_multi<N>(d);
}
__device__ __forceinline__ double dot_value(const FF &x) { return ff_value(x); }
__device__ __forceinline__ double dot_value(double x) { return x; }

// BATCH: the lattices of a batch in one launch (NR = 1; right-hand side k is lattice k).
// RG: groups of right-hand sides sharing a site's threads (dslash_item).
// WG > 1 (no epilogue, one thread per site, RG = 1): the block's threads form WG slices of
// a.bs threads over the same sites, slice g taking the g-th of the block's WG groups of NR
// right-hand sides; their link loads allocate in L1, so one L2 read of a link serves the
// block's WG NR right-hand sides without the registers of WG NR accumulators per thread.
template <int PL, int PV, int NREAL, int NR, int EPI, int DS, bool BATCH, int RG = 1, int WG = 1>
__global__ void __launch_bounds__(kDslashMaxBlock) k_dslash(const DslashArgs a)
{
    static_assert(WG == 1 || (EPI == 0 && DS == 1 && RG == 1 && !BATCH), "block slices: plain Dslash, one thread per site");
    using T = Prec<PV>;
    using TL = Prec<PL>;
    static_assert(std::is_same<typename T::Link, typename TL::Link>::value, "link and vector arithmetic must agree");
    static_assert(!BATCH || NR == 1, "batches take one right-hand side per lattice");
    if (a.skip) { // uniform over the grid: the scalars do not change during the launch
        bool any = false;
        for (int r = 0; r < a.nrhs; r++) any |= a.skip[r].active != 0;
        if (!any) {
            // A launch that carries the loop control (the single-reduction CG epilogue) still
            // closes the iteration: the iteration stamps advance as the finishing step would
            // advance them, so no earlier alpha counts as fresh for the update that follows,
            // and the device loop is told that nothing is active.
            if constexpr (EPI == 2) {
                if (a.red.partials && a.red.ctl && blockIdx.x == 0 && threadIdx.x == 0) {
                    for (int r = 0; r < a.nrhs; r++) a.red.sc[r].it_all++;
                    finish_control(a.red, a.nrhs);
                }
            }
            return;
        }
    }
    constexpr int ND = EpiDots<EPI>::n;
    // FP32 vectors: the epilogue's dot products in float-float pairs, float scales and m4
    // (no FP64 operation per site or per thread; one conversion per block and value)
    constexpr bool FFK = PV == HISQ_F32 && RG == 1;
    using DTK = std::conditional_t<FFK, FF, double>;
    DTK dots[NR * ND];
#pragma unroll
    for (int r = 0; r < NR * ND; r++) dots[r] = DTK{};
    if constexpr (BATCH) {
        // One block per tile; with the epilogue's reduction a resident grid whose blocks
        // stride over the tiles: each tile's dot products go to its own partial (the tile
        // number of its lattice), and a block arrives once, after its last tile, instead of
        // every tile paying the block sum's barriers and the arrival's round trip in a wave
        // of its own.
        __shared__ Geom sg;
        constexpr int d = DS == 1 ? 0 : DS == 2 ? 1 : 2;
        const BatchDesc &B = *a.batch;
        for (uint32_t item = blockIdx.x; item < a.items; item += gridDim.x) {
            int k = 0;
            while (k + 1 < B.n && B.tstart[d][k + 1] <= item) k++;
            const uint32_t tile = item - B.tstart[d][k];
            __syncthreads(); // the previous tile's readers of sg are done
            if (threadIdx.x == 0) sg = B.lat[k].g;
            __syncthreads();
            const size_t off = (size_t)k * a.rhs_bytes;
            const BatchLattice &L = B.lat[k];
            const auto sc0 = [&] { if constexpr (FFK) return L.scale_f[PL][0]; else return L.scale[PL][0]; }();
            const auto sc1 = [&] { if constexpr (FFK) return L.scale_f[PL][1]; else return L.scale[PL][1]; }();
            DTK td[ND];
#pragma unroll
            for (int j = 0; j < ND; j++) td[j] = DTK{};
            dslash_item<PL, PV, NREAL, 1, EPI, DS, false, false, 1, DTK>(
                a, sg, L.links[PL], L.slot_bytes[PL], sc0, sc1, a.in + off, a.out + off, EPI ? a.pv + off : nullptr,
                EPI == 2 ? a.rv + off : nullptr, a.shift ? a.shift + k : nullptr, tile, td);
            if constexpr (EPI >= 1) {
                if (a.red.partials) {
                    block_sum_dots<FFK, ND>(td);
                    if (threadIdx.x == 0) {
#pragma unroll
                        for (int j = 0; j < ND; j++)
                            a.red.partials[(size_t)(ND * k + j) * a.red.nblocks + tile] = dot_value(td[j]);
                        // partials of lattice k beyond its own tiles are zero
                        if (tile == 0)
                            for (int j = 0; j < ND; j++)
                                for (int i = (int)(B.tstart[d][k + 1] - B.tstart[d][k]); i < a.red.nblocks; i++)
                                    a.red.partials[(size_t)(ND * k + j) * a.red.nblocks + i] = 0.0;
                    }
                }
            }
        }
        if constexpr (EPI >= 1) {
            // the partials are in place: arrive (no values of its own), the last block finishes
            if (a.red.partials) grid_reduce<ND>(a.red, nullptr, 0, 0, ND * a.nrhs, 0);
        }
    } else {
        // gridDim.x is a multiple of the group count, so a block keeps one group of right-hand
        // sides while it strides over the work items (site tile, group)
        // (with WG slices, a block group is WG consecutive groups, slice g of the block taking
        // the g-th; a.bs is then the threads of one slice)
        const uint32_t ngroups = (uint32_t)(a.nrhs / (NR * RG * WG));
        const uint32_t slice = WG > 1 ? threadIdx.x / (uint32_t)a.bs : 0u;
        const uint32_t tid = WG > 1 ? threadIdx.x - slice * (uint32_t)a.bs : threadIdx.x;
        const int rhs0 = (int)((blockIdx.x % ngroups) * WG + slice) * NR * RG;
        const size_t off = (size_t)rhs0 * a.rhs_bytes;
        const auto sc0 = [&] { if constexpr (FFK) return a.scale_f[0]; else return a.scale[0]; }();
        const auto sc1 = [&] { if constexpr (FFK) return a.scale_f[1]; else return a.scale[1]; }();
        for (uint32_t item = blockIdx.x; item < a.items; item += gridDim.x)
            dslash_item<PL, PV, NREAL, NR, EPI, DS, false, false, RG, DTK, (WG > 1)>(
                a, a.g, a.links, a.slot_bytes, sc0, sc1, a.in + off, a.out + off, EPI ? a.pv + off : nullptr,
                EPI == 2 ? a.rv + off : nullptr, a.shift ? a.shift + rhs0 : nullptr, item / ngroups, dots, tid);
        if constexpr (EPI >= 1) {
            if (a.red.partials) { // uniform over the grid
                if constexpr (RG == 1) {
                    block_sum_dots<FFK, NR * ND>(dots);
                    double dd[NR * ND];
#pragma unroll
                    for (int j = 0; j < NR * ND; j++) dd[j] = threadIdx.x == 0 ? dot_value(dots[j]) : 0.0; // read on thread 0
                    grid_reduce<NR * ND>(a.red, dd, NR * ND, ND * rhs0, ND * a.nrhs, (int)(blockIdx.x / ngroups));
                } else {
                    const double *sums = block_sum_groups<NR * ND, RG>(dots);
                    grid_reduce<NR * ND>(a.red, sums, RG * NR * ND, ND * rhs0, ND * a.nrhs,
                                         (int)(blockIdx.x / ngroups));
                }
            }
        }
    }
}

// ---------------------------------------------------------------- launch table
// Work items are (site tile of kDslashBlock threads, group of NR right-hand sides), the
// group fastest.  Without a reduction every item is a block of its own.  With the
// epilogue's reduction the grid holds at most as many blocks as are resident at once (a
// multiple of the group count, from the occupancy of this instantiation) and blocks
// stride over the items, so that there is one partial per block and right-hand side.
template <int PL, int PV, int NREAL, int NR, int EPI, int DS, bool BATCH, int RG = 1, int WG = 1>
static cudaError_t launch_one(const DslashArgs &a0, cudaStream_t st)
{
    DslashArgs a = a0;
    const int bs = BATCH ? kDslashBlock : a.bs;
    if (bs != 64 && bs != 128 && bs != 256) return cudaErrorInvalidValue;
    a.bs = bs;
    static int occ[3] = {-1, -1, -1}; // resident blocks per SM of this instantiation, per block size
    const int bi = bs == 64 ? 0 : bs == 128 ? 1 : 2;
    if (occ[bi] < 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_dslash<PL, PV, NREAL, NR, EPI, DS, BATCH, RG, WG>, bs,
                                                          0) != cudaSuccess ||
            o < 1)
            o = 1;
        occ[bi] = o;
    }
    if constexpr (BATCH) { // one block per tile of every lattice; a resident grid with a reduction
        constexpr int d = DS == 1 ? 0 : DS == 2 ? 1 : 2;
        const uint32_t items = a.batch_tiles[d];
        const uint32_t resident = (uint32_t)std::max(1, a.sm_count) * (uint32_t)occ[bi];
        const uint32_t blocks = a.red.partials ? std::min(items, resident) : items;
        a.items = items;
        a.red.nblocks = (int)a.batch_maxtiles[d]; // partials per lattice (zero beyond its tiles)
        a.red.ntotal = (int)blocks;
        k_dslash<PL, PV, NREAL, 1, EPI, DS, true><<<blocks, kDslashBlock, 0, st>>>(a);
        return cudaGetLastError();
    } else {
        const int ts = bs / WG; // threads over the sites of one tile (one slice of the block)
        if (ts < 32) return cudaErrorInvalidValue;
        a.bs = ts;
        const size_t tiles = ((size_t)a.g.Vh * DS * RG + ts - 1) / ts;
        const size_t ng = (size_t)(a.nrhs / (NR * RG * WG));
        const size_t items = tiles * ng;
        const size_t resident = std::max<size_t>(ng, (size_t)std::max(1, a.sm_count) * occ[bi] / ng * ng);
        const size_t blocks = a.red.partials ? std::min(items, resident) : items;
        if (items > 0xffffffffull) return cudaErrorInvalidValue;
        a.items = (uint32_t)items;
        a.red.nblocks = (int)(blocks / ng); // partials per right-hand side
        a.red.ntotal = (int)blocks;
        k_dslash<PL, PV, NREAL, NR, EPI, DS, false, RG, WG><<<(unsigned)blocks, bs, 0, st>>>(a);
        return cudaGetLastError();
    }
}

template <int PL, int PV, int NREAL, int EPI, int DS>
static cudaError_t launch_nr(const DslashArgs &a, int nr, int rg, cudaStream_t st)
{
    if (a.nrhs < 1 || a.nrhs % (nr * rg)) return cudaErrorInvalidValue;
    if (a.batch) { // one right-hand side per lattice, storage order
        if (nr != 1 || rg != 1 || a.zt || a.nrhs != a.batch_n) return cudaErrorInvalidValue;
        return launch_one<PL, PV, NREAL, 1, EPI, DS, true>(a, st);
    }
    if (a.zt && !a.g.zt_ok) return cudaErrorInvalidValue;
    if (a.wg > 1) { // slices of a block over the same sites: plain Dslash, one thread per site
        if constexpr (EPI == 0 && DS == 1) {
            if (rg == 1 && a.nrhs % (nr * a.wg) == 0) {
                switch (a.wg * 16 + nr) {
                case 2 * 16 + 1: return launch_one<PL, PV, NREAL, 1, 0, 1, false, 1, 2>(a, st);
                case 2 * 16 + 2: return launch_one<PL, PV, NREAL, 2, 0, 1, false, 1, 2>(a, st);
                case 2 * 16 + 4: return launch_one<PL, PV, NREAL, 4, 0, 1, false, 1, 2>(a, st);
                case 4 * 16 + 1: return launch_one<PL, PV, NREAL, 1, 0, 1, false, 1, 4>(a, st);
                case 4 * 16 + 2: return launch_one<PL, PV, NREAL, 2, 0, 1, false, 1, 4>(a, st);
                case 4 * 16 + 4: return launch_one<PL, PV, NREAL, 4, 0, 1, false, 1, 4>(a, st);
                }
            }
        }
        return cudaErrorInvalidValue;
    }
    if (rg != 1) { // groups of right-hand sides on one site's threads: one thread per site only
        if constexpr (DS == 1) {
            switch (rg * 16 + nr) {
            case 2 * 16 + 1: return launch_one<PL, PV, NREAL, 1, EPI, 1, false, 2>(a, st);
            case 2 * 16 + 2: return launch_one<PL, PV, NREAL, 2, EPI, 1, false, 2>(a, st);
            case 2 * 16 + 4: return launch_one<PL, PV, NREAL, 4, EPI, 1, false, 2>(a, st);
            case 4 * 16 + 1: return launch_one<PL, PV, NREAL, 1, EPI, 1, false, 4>(a, st);
            case 4 * 16 + 2: return launch_one<PL, PV, NREAL, 2, EPI, 1, false, 4>(a, st);
            case 4 * 16 + 4: return launch_one<PL, PV, NREAL, 4, EPI, 1, false, 4>(a, st);
            }
        }
        return cudaErrorInvalidValue;
    }
    switch (nr) {
    case 1: return launch_one<PL, PV, NREAL, 1, EPI, DS, false>(a, st);
    case 2: return launch_one<PL, PV, NREAL, 2, EPI, DS, false>(a, st);
    case 4: return launch_one<PL, PV, NREAL, 4, EPI, DS, false>(a, st);
    case 8:
        if constexpr (PV == HISQ_F64 || PV == HISQ_F64X) return cudaErrorInvalidValue;
        else return launch_one<PL, PV, NREAL, 8, EPI, DS, false>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int PL, int PV, int NREAL, int EPI>
static cudaError_t launch_ds(const DslashArgs &a, int nr, int ds, int rg, cudaStream_t st)
{
    switch (ds) {
    case 1: return launch_nr<PL, PV, NREAL, EPI, 1>(a, nr, rg, st);
    case 2: return launch_nr<PL, PV, NREAL, EPI, 2>(a, nr, rg, st);
    case 4: return launch_nr<PL, PV, NREAL, EPI, 4>(a, nr, rg, st);
    }
    return cudaErrorInvalidValue;
}

template <int PL, int PV, int EPI>
static cudaError_t launch_prec(const DslashArgs &a, int nreal, int nr, int ds, int rg, cudaStream_t st)
{
    if (nreal == 12) {
        if constexpr (PL == HISQ_F64X) return cudaErrorInvalidValue;
        else return launch_ds<PL, PV, 12, EPI>(a, nr, ds, rg, st);
    }
    return launch_ds<PL, PV, 18, EPI>(a, nr, ds, rg, st);
}

// instantiate the launcher of one link precision with one vector precision
// (the CG epilogue, EPI = 2, exists for the vector precisions a solver iterates: not 16-bit)
#define HISQ_DSLASH_INSTANTIATE(PL, PV)                                                                  \
    cudaError_t dslash_launch_##PL##_##PV(int epi, const DslashArgs &a, int nreal, int nr, int ds, int rg, \
                                          cudaStream_t st)                                               \
    {                                                                                                    \
        if (epi == 2) {                                                                                  \
            if constexpr (PV == HISQ_F16 || PV == HISQ_BF16) return cudaErrorInvalidValue;              \
            else return launch_prec<PL, PV, 2>(a, nreal, nr, ds, rg, st);                                 \
        }                                                                                                \
        return epi ? launch_prec<PL, PV, 1>(a, nreal, nr, ds, rg, st)                                    \
                   : launch_prec<PL, PV, 0>(a, nreal, nr, ds, rg, st);                                   \
    }

}  // namespace hisq
