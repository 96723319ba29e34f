// dslash_kernel.cuh -- the HISQ staggered Dslash (Sec. 5.1) on one parity, all storage precisions.
//
//   out(x) = sum_mu [ X_mu(x) phi(x+mu) - X_mu(x-mu)^+ phi(x-mu)
//                   + W_mu(x) phi(x+3mu) - W_mu(x-3mu)^+ phi(x-3mu) ]      (x of parity p)
// with the staggered phases and the antiperiodic time boundary folded into the stored
// links (18 reals) or applied here (12 reals: rows 0 and 1 carry the sign, row 2 is
// rebuilt and signed in registers).
//
// One thread computes one output site for NR right-hand sides (the paper's N_inner loop,
// Sec. 5.1), so every link is loaded once per NR vectors; grid.y runs over groups of NR
// right-hand sides (N_outer), adjacent in launch order so the second group finds the
// links in L2.  Links stream through with L1-bypassing 16-byte loads (read once per
// application); neighbour spinors are gathered through L1/L2, where their 16-fold reuse
// happens.  Optional epilogue (normal operator, Sec. 3.2 applyMdaggM):
//   out = m4 * p - D in,   and <p, out> reduced in FP64 per right-hand side.
#pragma once

#include "arith.cuh"
#include "dslash.cuh"
#include "reduce.cuh"

namespace hisq {

template <int P, int NREAL, int NR, int EPI>
__global__ void __launch_bounds__(kDslashBlock) k_dslash(const DslashArgs a)
{
    using T = Prec<P>;
    constexpr int LB = NREAL == 18 ? LinkBytes<P>::b18 : LinkBytes<P>::b12;
    constexpr bool TWO = (P == HISQ_F16 || P == HISQ_BF16 || NREAL == 12);
    if (a.skip) { // uniform over the grid: the scalars do not change during the launch
        bool any = false;
        for (int r = 0; r < a.nrhs; r++) any |= a.skip[r].active != 0;
        if (!any) return;
    }
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs0 = blockIdx.y * NR;
    double dots[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) dots[r] = 0.0;

    if (s < a.g.Vh) {
        const Site c = site_coords(a.g, s, a.p);
        typename T::Acc acc[TWO ? 2 : 1][NR];
#pragma unroll
        for (int t = 0; t < (TWO ? 2 : 1); t++)
#pragma unroll
            for (int r = 0; r < NR; r++) T::zero(acc[t][r]);

        constexpr bool SPLIT = T::kSplitDirections;
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            typename T::Acc dacc[SPLIT ? NR : 1];
            if constexpr (SPLIT) {
#pragma unroll
                for (int r = 0; r < NR; r++) T::zero(dacc[r]);
            }
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const int k = h == 0 ? 1 : h == 1 ? -1 : h == 2 ? 3 : -3;
                const int type = h >> 1;
                const bool back = h & 1;
                bool wrap;
                const uint32_t sn = neighbour(a.g, c, s, mu, k, wrap);
                const int lp = back ? 1 - a.p : a.p;
                const char *slot = a.links + (size_t)((lp * 2 + type) * 4 + mu) * a.slot_bytes;
                uint32_t w[LB / 4];
                load_link_words<LB>(slot, back ? sn : s, w);
                typename T::Link U;
                T::template unpack<NREAL>(w, U);
                if constexpr (NREAL == 12) T::rebuild(U, (eta_neg(c, mu) != 0) ^ (mu == 3 && wrap));
#pragma unroll
                for (int r = 0; r < NR; r++) {
                    typename T::Vec v;
                    T::load(a.in + (size_t)(rhs0 + r) * a.rhs_bytes, sn, v);
                    typename T::Acc &dst = SPLIT ? dacc[SPLIT ? r : 0] : acc[TWO ? type : 0][r];
                    if (back) T::template hop<true, true>(dst, U, v);
                    else T::template hop<false, false>(dst, U, v);
                }
            }
            if constexpr (SPLIT) {
#pragma unroll
                for (int r = 0; r < NR; r++) {
                    if (mu == 0) acc[0][r] = dacc[r];
                    else T::add_acc(acc[0][r], dacc[r]);
                }
            }
        }

#pragma unroll
        for (int r = 0; r < NR; r++) {
            typename T::Acc o;
            if constexpr (TWO) {
                T::zero(o);
                T::axpy_acc(o, (typename T::Real)a.scale[0], acc[0][r]);
                T::axpy_acc(o, (typename T::Real)a.scale[1], acc[1][r]);
            } else {
                o = acc[0][r];
            }
            if constexpr (EPI == 1) {
                typename T::Vec pv;
                T::load(a.pv + (size_t)(rhs0 + r) * a.rhs_bytes, s, pv);
                T::mdagm_epilogue(o, a.m4, pv);
                dots[r] = T::dot(pv, o);
            }
            T::store(a.out + (size_t)(rhs0 + r) * a.rhs_bytes, s, o);
        }
    }
    if constexpr (EPI == 1) {
        if (a.red.partials) { // uniform over the grid
            double mine[NR];
#pragma unroll
            for (int r = 0; r < NR; r++) mine[r] = block_sum(dots[r]);
            grid_reduce<NR>(a.red, mine, NR, rhs0, a.nrhs, blockIdx.x);
        }
    }
}

// ---------------------------------------------------------------- launch table
template <int P, int NREAL, int EPI>
static cudaError_t launch_nr(const DslashArgs &a, int nr, cudaStream_t st)
{
    dim3 grid((a.g.Vh + kDslashBlock - 1) / kDslashBlock, a.nrhs / nr);
    switch (nr) {
    case 1: k_dslash<P, NREAL, 1, EPI><<<grid, kDslashBlock, 0, st>>>(a); break;
    case 2: k_dslash<P, NREAL, 2, EPI><<<grid, kDslashBlock, 0, st>>>(a); break;
    case 4: k_dslash<P, NREAL, 4, EPI><<<grid, kDslashBlock, 0, st>>>(a); break;
    case 8: k_dslash<P, NREAL, 8, EPI><<<grid, kDslashBlock, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int P, int EPI>
static cudaError_t launch_prec(const DslashArgs &a, int nreal, int nr, cudaStream_t st)
{
    if (nreal == 12) {
        if constexpr (P == HISQ_F64X) return cudaErrorInvalidValue;
        else return launch_nr<P, 12, EPI>(a, nr, st);
    }
    return launch_nr<P, 18, EPI>(a, nr, st);
}

// instantiate the launcher of one precision (one translation unit per precision)
#define HISQ_DSLASH_INSTANTIATE(P)                                                               \
    cudaError_t dslash_launch_##P(int epi, const DslashArgs &a, int nreal, int nr, cudaStream_t st) \
    {                                                                                            \
        return epi ? launch_prec<P, 1>(a, nreal, nr, st) : launch_prec<P, 0>(a, nreal, nr, st);   \
    }

}  // namespace hisq
