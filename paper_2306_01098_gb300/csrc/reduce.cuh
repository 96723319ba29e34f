// reduce.cuh -- deterministic grid reductions with a "last block finishes" step, and the
// per-right-hand-side scalars of the CG recurrences kept on the device.
//
// Each block writes one FP64 partial per value; the block that arrives last (atomic
// counter after a fence) sums the partials of every value in a fixed order and applies a
// finishing operation, so no host round trip or extra launch is needed between the
// reduction and the scalar recurrences that consume it.
#pragma once

#include "internal.cuh"

namespace hisq {

// scalars of one right-hand side / shift, device resident
struct Scalars {
    double rr;      // |r|^2 of the current residual
    double pAp;     // <p, A p>
    double alpha;   // rr / pAp
    double beta;    // rr_new / rr
    double stop;    // sloppy stopping threshold on |r|^2
    double rr_ref;  // |r|^2 at the last reliable update
    double delta2;  // reliable-update trigger: rr < delta2 * rr_ref
    double last;    // scratch: last reduced value
    double bb;      // |b|^2
    int iters;      // iterations performed while active
    int it_all;     // iterations launched (advanced by every |r|^2 reduction)
    int astamp;     // it_all of the iteration whose <p,Ap> produced alpha
    int active;     // 1 while iterating
    int paused;     // 1: stopped for a reliable update (sloppy residual fell below delta)
    double last_im; // scratch: imaginary part of the last reduced complex value
    int flag;       // 1: reliable update wanted (sloppy target or delta reached)
    int bad;        // 1: non-finite or non-positive curvature seen
    int pad;
};

// alpha is consumed only in the iteration that produced it: the residual update requires
// astamp == it_all (before the |r|^2 reduction advances it_all), the solution update
// astamp == it_all - 1.  When every right-hand side has converged the operator launches
// return at once, alpha is not refreshed, and the stamps keep the updates from reusing it.
__device__ __forceinline__ bool alpha_fresh_for_r(const Scalars &S) { return S.active && S.astamp == S.it_all; }
__device__ __forceinline__ bool alpha_fresh_for_x(const Scalars &S) { return S.astamp == S.it_all - 1; }

enum FinishOp {
    FIN_STORE = 0, // last = total
    FIN_ALPHA = 1, // pAp = total; alpha = rr / pAp
    FIN_RR = 2,    // beta = total / rr; rr = total; set flag when below stop / delta
    FIN_CDOT = 3,  // value 2k -> last, 2k+1 -> last_im of right-hand side k
    FIN_AB = 4,    // values 4k .. 4k+3 = <p,Ap>, |r|^2, <r,Ap>, <Ap,Ap> of right-hand side k:
                   // alpha = |r|^2 / <p,Ap> (curvature checked as FIN_ALPHA), then
                   // |r - alpha Ap|^2 = |r|^2 - 2 alpha <r,Ap> + alpha^2 <Ap,Ap> and
                   // everything FIN_RR does with it.  |r|^2 is reduced afresh from the stored
                   // r each iteration, so the rounding of the expansion does not accumulate.
};

// iteration control of a device-side solver loop (a CUDA graph WHILE node): the block that
// finishes the |r|^2 reduction also decides whether the loop goes on
struct LoopCtl {
    int start; // it_all when the phase began
    int cap;   // iterations allowed in this phase
    int mode;  // for the x/p update of this iteration: 0 = x and p, 1 = x only (last iteration)
    int pad;
};

struct Reduce {
    LoopCtl *ctl = nullptr;               // if set: decide continuation after finishing
    unsigned long long cond = 0;          // graph conditional handle (0: not inside a graph)
    double *partials = nullptr; // [nval][nblocks]
    unsigned *counter = nullptr;
    Scalars *sc = nullptr;      // nval scalars (indexed from sc_offset)
    int op = FIN_STORE;
    int nblocks = 0;            // partials per value (blocks along grid x)
    int ntotal = 0;             // blocks in the grid (all must arrive before finishing)
};

// alpha = rr / <p,Ap> from the reduced curvature (FIN_ALPHA)
__device__ __forceinline__ void fin_alpha(Scalars &S, double total)
{
    S.pAp = total;
    S.astamp = S.it_all;
    if (S.active && !(total > 0.0 && isfinite(total))) {
        S.bad = 1;
        S.active = 0;
    }
    S.alpha = S.active ? S.rr / total : 0.0;
}

// the new |r|^2 has been reduced (FIN_RR): beta, the iteration stamps and the stop/pause flags
__device__ __forceinline__ void fin_rr(Scalars &S, double total)
{
    S.it_all++;
    if (S.active) {
        S.iters++;
        if (!isfinite(total)) {
            S.bad = 1;
            S.active = 0;
            S.beta = 0.0;
            return;
        }
        S.beta = S.rr > 0.0 ? total / S.rr : 0.0;
        S.rr = total;
        // the sloppy residual may not run ahead of the true one: at the target, or a
        // factor delta below the last recomputed residual, the right-hand side pauses
        // until the host's reliable update (delta2 = 0 for plain FP64 solves)
        if (total <= S.stop || total < S.delta2 * S.rr_ref) {
            S.flag = 1;
            S.active = 0;
            S.paused = total > S.stop;
        }
    }
    // an inactive right-hand side keeps beta: a reliable update after a pause needs it
}

// single-reduction step (FIN_AB) once S.pAp = <p,Ap>, S.last_im = |r|^2 (of the stored r) and
// S.last = <r,Ap> are in place and ApAp = <Ap,Ap>: alpha, then
// |r - alpha Ap|^2 = |r|^2 - 2 alpha <r,Ap> + alpha^2 <Ap,Ap> and everything FIN_RR does with it
__device__ __forceinline__ void fin_ab(Scalars &S, double ApAp)
{
    if (S.active && isfinite(S.last_im)) S.rr = S.last_im;
    const double pAp = S.pAp;
    S.astamp = S.it_all;
    if (S.active && !(pAp > 0.0 && isfinite(pAp))) {
        S.bad = 1;
        S.active = 0;
    }
    S.alpha = S.active ? S.rr / pAp : 0.0;
    double rr = S.rr;
    if (S.active) {
        rr = S.rr - 2.0 * S.alpha * S.last + S.alpha * S.alpha * ApAp;
        if (isfinite(rr) && rr < 0.0) rr = 0.0; // rounding: the residual has vanished
    }
    fin_rr(S, rr);
}

__device__ __forceinline__ void finish_value(const Reduce &R, int v, double total)
{
    Scalars &S = R.sc[R.op == FIN_CDOT ? (v >> 1) : R.op == FIN_AB ? (v >> 2) : v];
    switch (R.op) {
    case FIN_AB:
        switch (v & 3) {
        case 0: S.pAp = total; return;     // <p, Ap>
        case 1: S.last_im = total; return; // |r|^2 of the stored r
        case 2: S.last = total; return;    // <r, Ap>
        default: fin_ab(S, total); return; // <Ap, Ap>: finish
        }
    case FIN_ALPHA: fin_alpha(S, total); break;
    case FIN_RR: fin_rr(S, total); break;
    case FIN_CDOT:
        if (v & 1) R.sc[v >> 1].last_im = total;
        else R.sc[v >> 1].last = total;
        break;
    default:
        S.last = total;
        break;
    }
}

// block-wide sum of one double; result valid on thread 0
__device__ __forceinline__ double block_sum(double x)
{
    __shared__ double wsum[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) wsum[w] = x;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = l < nw ? wsum[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

// loop control after the final sums (thread 0); nrhs = right-hand sides (scalars)
__device__ __forceinline__ void finish_control(const Reduce &R, int nrhs)
{
    if (R.ctl) {
        bool any = false;
        for (int v = 0; v < nrhs; v++) any |= R.sc[v].active != 0;
        const bool last = R.sc[0].it_all - R.ctl->start >= R.ctl->cap;
        R.ctl->mode = last ? 1 : 0;
        if (R.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)R.cond, (any && !last) ? 1u : 0u);
    }
}

// ---------------------------------------------------------------- float-float sums
// A sum kept as an unevaluated pair of floats h + l, accumulated on the FP32 pipes: on this
// GPU an FP64 add or conversion costs about as much as sixty FP32 operations, and the dot
// products of the FP32 iteration vectors are summed over every site each iteration.
// Adding a float uses Knuth's TwoSum (the exact rounding error of h + x goes into l);
// merging two pairs is TwoSum on the high parts followed by Dekker's Fast2Sum
// renormalisation.  The explicit _rn intrinsics keep the compiler from contracting or
// reassociating the error terms.  The value is (double)h + (double)l, accurate to about
// 2^-44 relative for sums of non-negative terms and to the usual cancellation bound otherwise.
struct FF {
    float h, l;
};

__device__ __forceinline__ void ff_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void ff_add(FF &a, float x)
{
    float s, e;
    ff_two_sum(a.h, x, s, e);
    a.h = s;
    a.l = __fadd_rn(a.l, e);
}

__device__ __forceinline__ void ff_merge(FF &a, const FF &b)
{
    float s, e;
    ff_two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    a.h = __fadd_rn(s, e);
    a.l = __fsub_rn(e, __fsub_rn(a.h, s));
}

__device__ __forceinline__ double ff_value(const FF &a) { return (double)a.h + (double)a.l; }

// block-wide float-float sums of NV values at once (one barrier for all); valid on thread 0
template <int NV>
__device__ __forceinline__ void block_sum_ff(FF (&x)[NV])
{
    __shared__ FF wsum_ff[NV][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const FF y = {__shfl_down_sync(0xffffffffu, x[v].h, o), __shfl_down_sync(0xffffffffu, x[v].l, o)};
            ff_merge(x[v], y);
        }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0)
#pragma unroll
        for (int v = 0; v < NV; v++) wsum_ff[v][w] = x[v];
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            FF r = l < nw ? wsum_ff[v][l] : FF{0.f, 0.f};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const FF y = {__shfl_down_sync(0xffffffffu, r.h, o), __shfl_down_sync(0xffffffffu, r.l, o)};
                ff_merge(r, y);
            }
            x[v] = r;
        }
    }
}

// block-wide sums of NV doubles at once (one barrier for all); results valid on thread 0
template <int NV>
__device__ __forceinline__ void block_sum_multi(double (&x)[NV])
{
    __shared__ double wsum[NV][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int v = 0; v < NV; v++) x[v] += __shfl_down_sync(0xffffffffu, x[v], o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0)
#pragma unroll
        for (int v = 0; v < NV; v++) wsum[v][w] = x[v];
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            double r = l < nw ? wsum[v][l] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
            x[v] = r;
        }
    }
}

// Block sums of NV doubles per group of right-hand sides, the group of a thread being
// lane % RG (RG consecutive lanes share a site, each with its own right-hand sides): lanes of
// one group are summed across the warp (xor offsets 16 .. RG), then across the warps in a
// fixed order.  Result in shared memory, value v of group g at out[g * NV + v]; valid for
// every thread after the call.
template <int NV, int RG>
__device__ __forceinline__ const double *block_sum_groups(double (&x)[NV])
{
    __shared__ double ws[RG * NV][32];
    __shared__ double res[RG * NV];
#pragma unroll
    for (int o = 16; o >= RG; o >>= 1)
#pragma unroll
        for (int v = 0; v < NV; v++) x[v] += __shfl_xor_sync(0xffffffffu, x[v], o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l < RG)
#pragma unroll
        for (int v = 0; v < NV; v++) ws[l * NV + v][w] = x[v];
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < RG * NV; k++) {
            double r = l < nw ? ws[k][l] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
            if (l == 0) res[k] = r;
        }
    }
    __syncthreads();
    return res;
}

// Grid reduction of `nval_all` values.  Block (bx, by) supplies the block sums of values
// [vbase, vbase + nmine) (thread 0 reads them from `mine`, registers or shared memory) as
// partial number bx of each;
// the last of the R.ntotal blocks to arrive sums the R.nblocks partials of every value
// in a fixed order and applies R.op.  The counter is reset for the next use.  NV is the
// number of values a call site supplies at once (the tail does not depend on it).
template <int NV>
__device__ __forceinline__ void grid_reduce(const Reduce &R, const double *mine, int nmine, int vbase, int nval_all,
                                            int bx)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        for (int v = 0; v < nmine; v++) R.partials[(size_t)(vbase + v) * R.nblocks + bx] = mine[v];
        // the arrival is an acquire-release add: it publishes this block's partials and, in
        // the last block, makes every other block's visible
        unsigned prev;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(R.counter) : "memory");
        last = (prev == (unsigned)R.ntotal - 1);
    }
    __syncthreads();
    if (!last) return;
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    // One warp per scalar slot (the four values of FIN_AB, the two of FIN_CDOT, else one
    // value): the warp's lanes sum the value's partials in a fixed order (lane l takes
    // partials l, l + 32, ... four at a time, then a fixed shuffle tree) and lane 0 finishes
    // the slot's values in value order.  Right-hand sides are finished in parallel, so the
    // serial tail does not grow with their number; the order is the same in every run.
    const int per = R.op == FIN_AB ? 4 : R.op == FIN_CDOT ? 2 : 1;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    for (int u = w; u < nval_all / per; u += nw)
        for (int j = 0; j < per; j++) {
            const int v = u * per + j;
            const double *pv = R.partials + (size_t)v * R.nblocks;
            double acc = 0.0;
            for (int i0 = l; i0 < R.nblocks; i0 += 128) {
                double t[4];
#pragma unroll
                for (int q = 0; q < 4; q++) t[q] = i0 + 32 * q < R.nblocks ? __ldcg(pv + i0 + 32 * q) : 0.0;
                acc += (t[0] + t[1]) + (t[2] + t[3]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (l == 0) finish_value(R, v, acc);
        }
    __syncthreads(); // every slot finished before the loop control reads the flags
    if (threadIdx.x == 0) {
        finish_control(R, R.op == FIN_AB ? nval_all / 4 : R.op == FIN_CDOT ? nval_all / 2 : nval_all);
        __threadfence();
        *R.counter = 0u;
    }
}

}  // namespace hisq
