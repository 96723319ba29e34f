// solver.cuh -- device workspace of the Krylov solvers, cached on the context.
#pragma once

#include <vector>

#include "blas.cuh"
#include "reduce.cuh"

namespace hisq {

struct SolverWork {
    int nrhs = 0, ps = -1, pv = -1, px = -1, pp = -1; // sloppy links, sloppy vectors, accumulator, precise
    DslashShape shape;
    bool tuned = false;
    uint32_t Vh = 0;
    const uint32_t *vh_rhs = nullptr; // batches: each right-hand side's own half volume (device)
    size_t rbS = 0, rbX = 0, rb64 = 0, rbP = 0; // bytes per rhs: sloppy, accumulator, canonical F64, padded F64
    char *r = nullptr, *p = nullptr, *Ap = nullptr, *t = nullptr, *xlo = nullptr; // sloppy vectors
    char *b64 = nullptr, *x64 = nullptr, *rhi = nullptr, *Axhi = nullptr, *thi = nullptr; // FP64
    char *xx = nullptr, *tx = nullptr, *Axx = nullptr; // float-pair precise operator
    Scalars *sc = nullptr;
    Scalars *h_sc = nullptr; // pinned host copy
    double *partials = nullptr;
    unsigned *counter = nullptr;
    LoopCtl *ctl = nullptr;  // device-side loop control
    void *phase_slots = nullptr; // arrival records of the persistent phase kernel (kPhaseMaxBlocks)
    DevStatus *h_status = nullptr; // pinned host copy of the device error flag
    double *shift_buf = nullptr, *h_shift = nullptr; // per right-hand side shifts (device, pinned host)
    const double *shift = nullptr;                   // shift_buf when shifts are in use
    std::vector<double> shift_key, graph_shift;      // shifts the loop graph was captured with
    int nblk_vec = 0, nblk_dslash = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t ev_sc = nullptr; // the scalars' read-back of a pipelined persistent phase
    cudaGraphExec_t graph = nullptr;
    double graph_m = -1.0;
    bool graph_l2 = false;
    bool fused = true, graph_fused = true; // single-reduction iteration (this call, the captured graph)
    std::vector<cudaEvent_t> prof;
    std::vector<void *> allocs;

    void release();
    int alloc(hisq_ctx *ctx, char **ptr, size_t bytes);
    Reduce red(int op, int nblocks_per_value, int ntotal = 0) const;
    // sites the vector passes cover per right-hand side (a batch skips its padding)
    Len len() const { return Len(Vh, vh_rhs); }
};

int get_work(hisq_ctx *ctx, int nrhs, int ps, int pp, SolverWork **out);

}  // namespace hisq
