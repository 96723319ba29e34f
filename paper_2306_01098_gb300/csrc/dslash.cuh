// dslash.cuh -- arguments, launch entry and tuning of the Dslash kernels.
#pragma once

#include "internal.cuh"
#include "reduce.cuh"

namespace hisq {

constexpr int kDslashBlock = 128;    // threads per block of batches and the default shape
constexpr int kDslashMaxBlock = 256; // largest block size of the autotuner's search

struct DslashArgs {
    Geom g;
    int p;                 // output parity
    const char *links;     // link store (16 slots)
    size_t slot_bytes;
    double scale[2];       // per link type multiplier (16-bit storage, 12-real c)
    const char *in;        // input field, parity 1-p, right-hand side 0
    char *out;             // output field, parity p
    size_t rhs_bytes;      // bytes between right-hand sides
    int nrhs;
    const Scalars *skip;   // if set: return at once when no right-hand side is active
    // normal-operator epilogue: out = m4 * pv - D in, <pv, out> reduced; with the CG
    // epilogue (EPI = 2) also <rv, out> and <out, out>
    const char *pv;
    const char *rv;
    double m4;
    float m4f;             // m4 and the scales as floats: the persistent CG kernel's FP32 path
    float scale_f[2];
    const double *shift;   // optional per right-hand side addition to m4 (device)
    Reduce red;
    int zt;                // launch order with z and t interchanged (Geom::zt_ok required)
    int stream_links;      // link store larger than L2 can keep: load links evict-first
    int sm_count;          // SMs of the device (grid size)
    int bs;                // threads per block (64, 128 or 256; batches: kDslashBlock)
    int wg;                // slices of a block over the same sites (DslashShape::wg; 0 or 1: none)
    uint32_t items;        // work items of the launch (set by the launcher)
    // batch of lattices (NULL for one lattice): device table, lattices, and from the host
    // copy of the table the tiles of all lattices / of the largest, per threads per site
    const BatchDesc *batch;
    int batch_n;
    uint32_t batch_tiles[3], batch_maxtiles[3];
};

DslashArgs make_dslash_args(hisq_ctx *ctx, int prec, int out_parity, const void *in, void *out, int nrhs,
                            size_t rhs_bytes);
// pl: link storage precision, pv: vector precision (equal, or 16-bit links with FP32 vectors)
cudaError_t dslash_launch(int pl, int pv, int epi, const DslashArgs &a, int nreal, const DslashShape &sh,
                          cudaStream_t st);
// The launcher fills red.nblocks (partials per right-hand side, at most the site tiles of
// the launch) and red.ntotal (blocks) of an epilogue reduction.
// shape for (pl, pv, nrhs) on this context: measured once per key (autotuner) unless tuning
// is off or the stream is capturing, then a size-based default
DslashShape dslash_shape(hisq_ctx *ctx, int pl, int pv, int nrhs, const void *in, void *out, size_t rhs_bytes,
                         cudaStream_t st);
int pick_inner(int prec, int nrhs);

#define HISQ_DSLASH_DECLARE(PL, PV) \
    cudaError_t dslash_launch_##PL##_##PV(int epi, const DslashArgs &a, int nreal, int nr, int ds, int rg,      \
                                          cudaStream_t st);
HISQ_DSLASH_DECLARE(HISQ_F64, HISQ_F64)
HISQ_DSLASH_DECLARE(HISQ_F64X, HISQ_F64X)
HISQ_DSLASH_DECLARE(HISQ_F32, HISQ_F32)
HISQ_DSLASH_DECLARE(HISQ_F16, HISQ_F16)
HISQ_DSLASH_DECLARE(HISQ_F16, HISQ_F32)
HISQ_DSLASH_DECLARE(HISQ_BF16, HISQ_BF16)
HISQ_DSLASH_DECLARE(HISQ_BF16, HISQ_F32)

}  // namespace hisq
