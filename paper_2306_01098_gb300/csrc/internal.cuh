// internal.cuh -- definitions shared by the CUDA sources of the HISQ library.
//
// Data layout in device memory
//   Links: one store per built precision.  A store holds 16 slots, slot (p, type, mu) =
//   ((p * 2 + type) * 4 + mu), type 0 = fat X, 1 = long W, p = parity of the site that
//   owns the link (the link U_mu(x) belongs to x).  Inside a slot the links of the Vh
//   sites of parity p are stored in blocks of 32 sites: block b holds, for its 32 lanes,
//   16-byte chunk q of every lane contiguously (32 x 16 B), chunk after chunk, followed
//   by the lane-contiguous tail (4 or 8 bytes per lane) when the link size is not a
//   multiple of 16.  A warp reading one chunk of 32 consecutive sites therefore reads
//   512 contiguous bytes.
//   Spinors (internal fields): site-major, one record per half-lattice site:
//     F64  : 6 doubles (re, im of 3 colours)                48 B
//     F64X : 6 hi floats then 6 lo floats                    48 B
//     F32  : 6 floats                                        24 B
//     F16/BF16 : 6 halves + one float scale                  16 B
//   Multi-RHS fields are [nrhs][VhPad] records.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>

#include "hisq.h"

namespace hisq {

constexpr int kFat = 0, kLong = 1;
constexpr int kSlots = 16;

// ---------------------------------------------------------------- fast integer division
// Division by a run-time invariant via multiply-high (Granlund & Montgomery, PLDI 1994):
// for 1 <= d < 2^31 and n < 2^31, q = (umulhi(n, m) + n) >> l with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1.
struct FastDiv {
    uint32_t d, m, l;
    __host__ void init(uint32_t div)
    {
        d = div;
        l = 0;
        while ((1ull << l) < div) l++;
        m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1);
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(n, m) + n) >> l; }
};

// ---------------------------------------------------------------- lattice geometry
struct Geom {
    int n[4];           // Nx, Ny, Nz, Nt
    int nxh;            // Nx / 2
    uint32_t Vh;        // half volume
    uint32_t VhPad;     // Vh rounded up to a multiple of 128
    uint32_t sy, sz, st;// half-index strides of y, z, t: nxh, nxh Ny, nxh Ny Nz
    FastDiv dx, dy, dz; // divide by nxh, Ny, Nz
    FastDiv dp, dt;     // divide by nxh Ny (sites of one z-t plane), Nt
    int zt_ok;          // the z-t interchanged site order is available (planes of whole warps, Nt < Nz)
};

struct Site {
    int x, y, z, t;
    uint32_t row; // half index of x = 0 (or 1) in this row: s - x/2
};

// coordinates of half-site s of parity p
__device__ __forceinline__ Site site_coords(const Geom &g, uint32_t s, int p)
{
    Site c;
    uint32_t r = g.dx.div(s);
    uint32_t xh = s - r * g.nxh;
    uint32_t q = g.dy.div(r);
    c.y = r - q * g.n[1];
    c.t = g.dz.div(q);
    c.z = q - c.t * g.n[2];
    c.x = 2 * xh + ((p + c.y + c.z + c.t) & 1);
    c.row = s - xh;
    return c;
}

// half index of the site k steps from c along mu (periodic), and whether the hop wrapped
__device__ __forceinline__ uint32_t neighbour(const Geom &g, const Site &c, uint32_t s, int mu, int k,
                                              bool &wrap)
{
    int v, n;
    switch (mu) {
    case 0: {
        n = g.n[0];
        v = c.x + k;
        wrap = (v < 0) | (v >= n);
        v += (v < 0) ? n : 0;
        v -= (v >= n) ? n : 0;
        return c.row + (v >> 1);
    }
    case 1:
        n = g.n[1];
        v = c.y + k;
        wrap = (v < 0) | (v >= n);
        v += (v < 0) ? n : 0;
        v -= (v >= n) ? n : 0;
        return s + (v - c.y) * (int)g.sy;
    case 2:
        n = g.n[2];
        v = c.z + k;
        wrap = (v < 0) | (v >= n);
        v += (v < 0) ? n : 0;
        v -= (v >= n) ? n : 0;
        return s + (v - c.z) * (int)g.sz;
    default:
        n = g.n[3];
        v = c.t + k;
        wrap = (v < 0) | (v >= n);
        v += (v < 0) ? n : 0;
        v -= (v >= n) ? n : 0;
        return s + (v - c.t) * (int)g.st;
    }
}

// MILC staggered phase eta_mu(x) as a sign bit (1 = negative)
__device__ __forceinline__ int eta_neg(const Site &c, int mu)
{
    switch (mu) {
    case 0: return 0;
    case 1: return c.x & 1;
    case 2: return (c.x + c.y) & 1;
    default: return (c.x + c.y + c.z) & 1;
    }
}

// ---------------------------------------------------------------- link store
template <int P> struct LinkBytes;
template <> struct LinkBytes<HISQ_F64>  { static constexpr int b18 = 144, b12 = 96; };
template <> struct LinkBytes<HISQ_F64X> { static constexpr int b18 = 144, b12 = 96; };
template <> struct LinkBytes<HISQ_F32>  { static constexpr int b18 = 72,  b12 = 48; };
template <> struct LinkBytes<HISQ_F16>  { static constexpr int b18 = 36,  b12 = 24; };
template <> struct LinkBytes<HISQ_BF16> { static constexpr int b18 = 36,  b12 = 24; };

__host__ __device__ inline int link_bytes(int prec, int nreal)
{
    switch (prec) {
    case HISQ_F64: case HISQ_F64X: return nreal * 8;
    case HISQ_F32: return nreal * 4;
    default: return nreal * 2;
    }
}

// vector storage used with a link precision by the canonical-layout entry points and the
// solvers: 16-bit links work on FP32 vectors (16-bit iteration vectors lose A-conjugacy at
// light masses and stall the solve); the 16-bit spinor format is used through fields
__host__ __device__ inline int vector_prec(int pl) { return (pl == HISQ_F16 || pl == HISQ_BF16) ? HISQ_F32 : pl; }

__host__ __device__ inline int spinor_bytes(int prec)
{
    switch (prec) {
    case HISQ_F64: case HISQ_F64X: return 48;
    case HISQ_F32: return 24;
    default: return 16;
    }
}

// byte offset of chunk q (16 B) / the tail of site s inside a slot with link size LB
__device__ __forceinline__ size_t link_chunk_off(uint32_t s, int LB, int q)
{
    return (size_t)(s >> 5) * (32 * LB) + q * 512 + (s & 31) * 16;
}
__device__ __forceinline__ size_t link_tail_off(uint32_t s, int LB, int tb)
{
    return (size_t)(s >> 5) * (32 * LB) + (LB / 16) * 512 + (s & 31) * tb;
}

struct LinkStore {
    char *base = nullptr;   // 16 slots
    size_t slot_bytes = 0;  // VhPad * link bytes
    int nreal = 0;          // 18 or 12
    int built = 0;
    double scale[2] = {1.0, 1.0}; // multiply the stored link by this (per type): 12-real c,
                                  // 16-bit max |entry|, else 1
};

// ---------------------------------------------------------------- device status
struct DevStatus {
    int error;      // device error flag (HISQ_EDEVICE when set)
    int where;
};

struct SolverWork;
struct MsWork;
struct FcgWork;

// Dslash launch shape: right-hand sides per thread (N_inner) and threads per site
struct DslashShape {
    int nr = 1;
    int ds = 1;
    int order = 0; // 0: sites in storage order (t slowest); 1: z and t interchanged in launch order
    int bs = 128;  // threads per block (sites per block = bs / (ds rg))
    int rg = 1;    // groups of right-hand sides sharing one site's threads (ds = 1 only)
    int wg = 1;    // groups of right-hand sides in one block, one slice of threads each, over the
                   // same sites (links shared through L1; plain Dslash, ds = 1, rg = 1 only)
};

// key of a Dslash shape in the context's tuning table: link precision, vector precision and
// the right-hand side count each in a field of its own, so no two keys collide
inline long long tune_key(int pl, int pv, int nrhs) { return ((long long)(pl * 8 + pv) << 32) | (unsigned)nrhs; }

// ---------------------------------------------------------------- batches of lattices
constexpr int kMaxBatch = 32;

// one lattice of a batch: its geometry and the link stores of its context
struct BatchLattice {
    Geom g;
    const char *links[HISQ_NPREC];
    size_t slot_bytes[HISQ_NPREC];
    double scale[HISQ_NPREC][2];
    float scale_f[HISQ_NPREC][2]; // the same as floats (FP32-vector kernels)
};

// Device table of a batch.  Work items of one launch are the site tiles of every lattice
// in turn: lattice k owns items [tstart[d][k], tstart[d][k + 1]) at 2^d threads per site.
// The vectors of lattice k start at right-hand side k of the padded solver layout.
struct BatchDesc {
    int n;
    uint32_t tstart[3][kMaxBatch + 1];
    uint32_t maxtiles[3]; // most tiles of one lattice
    uint32_t vh[kMaxBatch]; // half volume of each lattice (the sites of its right-hand side)
    BatchLattice lat[kMaxBatch];
};

}  // namespace hisq

// ---------------------------------------------------------------- context and fields
struct hisq_ctx {
    int device = 0;
    int sm_count = 0;
    size_t l2_persist_max = 0; // largest persisting L2 carve-out (bytes)
    int dims[4] = {0, 0, 0, 0};
    hisq::Geom g{};
    int links_phased = 0;
    int autotune = 1;
    std::map<long long, hisq::DslashShape> tune; // autotuned Dslash shapes, keyed by hisq::tune_key
    hisq::LinkStore links[HISQ_NPREC];
    int last_error = 0;
    std::string msg;
    // scratch owned by the context (grown on demand)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    hisq::DevStatus *status = nullptr;
    hisq::SolverWork *solver = nullptr; // cached solver workspace
    hisq::MsWork *msolver = nullptr;    // cached multi-shift workspace
    hisq::FcgWork *fcg = nullptr;       // cached flexible-CG workspace
    // a context that stands for a batch of lattices (hisq_batch): device and host tables;
    // its Vh is the largest member's, its link stores belong to the members
    hisq::BatchDesc *batch = nullptr;
    hisq::BatchDesc *batch_host = nullptr;
};

struct hisq_field {
    hisq_ctx *ctx = nullptr;
    int prec = 0;
    int nrhs = 0;
    size_t rhs_bytes = 0; // bytes per right-hand side (VhPad * spinor bytes)
    void *data = nullptr;
};

namespace hisq {

int set_error(hisq_ctx *ctx, int code, const std::string &msg);
int cuda_error(hisq_ctx *ctx, cudaError_t e, const char *what);
int ensure_workspace(hisq_ctx *ctx, size_t bytes);
void release_work(hisq_ctx *ctx);
void release_ms_work(hisq_ctx *ctx);
void release_fcg_work(hisq_ctx *ctx);

#define HISQ_CUDA(ctx, call)                                      \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return hisq::cuda_error((ctx), e_, #call); \
    } while (0)

// launch helpers implemented in the .cu files
int launch_dslash2(hisq_ctx *ctx, int pl, int pv, int out_parity, const void *in, void *out, int nrhs,
                   size_t rhs_bytes, cudaStream_t st);
int launch_dslash(hisq_ctx *ctx, int prec, int out_parity, const void *in, void *out, int nrhs,
                  size_t rhs_bytes, cudaStream_t st);
int launch_import(hisq_ctx *ctx, int prec, const double *src, void *dst, int nrhs, size_t rhs_bytes,
                  cudaStream_t st);
int launch_export(hisq_ctx *ctx, int prec, const void *src, double *dst, int nrhs, size_t rhs_bytes,
                  cudaStream_t st);

}  // namespace hisq
