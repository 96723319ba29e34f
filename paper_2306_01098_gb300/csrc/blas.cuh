// blas.cuh -- fused vector kernels of the Krylov solvers (one pass over each vector).
//
// Vectors are internal-layout fields (VecRef: base + bytes between right-hand sides);
// grid.y runs over right-hand sides, grid.x is a fixed number of blocks looping over
// sites, so every reduction has a fixed partial count and a fixed summation order.
// Reductions accumulate per thread in the compute type of the field, per block and grid
// in FP64.  Kernels skip right-hand sides whose coefficients are zero (converged).
#pragma once

#include "arith.cuh"
#include "reduce.cuh"

namespace hisq {

constexpr int kVecBlock = 256;

struct VecRef {
    char *p;
    size_t rb; // bytes between right-hand sides
    __device__ __forceinline__ char *rhs(int r) const { return p + (size_t)r * rb; }
};

// Sites of each right-hand side: Vh for all of them, or, for a batch of lattices padded to
// its largest member (per != nullptr, device memory), right-hand side r's own half volume
// per[r], so that the vector passes never touch the padding.
struct Len {
    uint32_t Vh;
    const uint32_t *per;
    __host__ __device__ Len(uint32_t vh, const uint32_t *p = nullptr) : Vh(vh), per(p) {}
    __device__ __forceinline__ uint32_t n(int rhs) const { return per ? per[rhs] : Vh; }
};

// ---------------------------------------------------------------- element operations
// y += a x ; y = x + b y ; |x|^2 ; conversions via double components
template <int P> struct Blas {
    using T = Prec<P>;
    using Vec = typename T::Vec;
    __device__ static void axpy(Vec &y, double a, const Vec &x)
    {
        const typename T::Real ar = (typename T::Real)a;
#pragma unroll
        for (int i = 0; i < 6; i++) y.v[i] = ar * x.v[i] + y.v[i];
    }
    __device__ static void xpay(Vec &y, const Vec &x, double b)
    {
        const typename T::Real br = (typename T::Real)b;
#pragma unroll
        for (int i = 0; i < 6; i++) y.v[i] = br * y.v[i] + x.v[i];
    }
    // y = a x + b y
    __device__ static void axpby(Vec &y, double a, const Vec &x, double b)
    {
        const typename T::Real ar = (typename T::Real)a, br = (typename T::Real)b;
#pragma unroll
        for (int i = 0; i < 6; i++) y.v[i] = ar * x.v[i] + br * y.v[i];
    }
    __device__ static double norm2(const Vec &x)
    {
        typename T::Real s = 0;
#pragma unroll
        for (int i = 0; i < 6; i++) s += x.v[i] * x.v[i];
        return (double)s;
    }
    __device__ static void store(char *base, uint32_t s, const Vec &x)
    {
        typename T::Acc a;
#pragma unroll
        for (int i = 0; i < 6; i++) a.v[i] = x.v[i];
        T::store(base, s, a);
    }
    __device__ static double get(const Vec &x, int i) { return (double)x.v[i]; }
    __device__ static void set(Vec &x, int i, double d) { x.v[i] = (typename T::Real)d; }
};

// float pairs: compensated updates on the FP32 pipes
template <> struct Blas<HISQ_F64X> {
    using T = Prec<HISQ_F64X>;
    using Vec = T::Vec;
    __device__ static void axpy(Vec &y, double a, const Vec &x)
    {
        const float ah = (float)a, al = (float)(a - (double)ah);
#pragma unroll
        for (int i = 0; i < 6; i++) {
            DAcc c = {y.h[i], y.l[i]};
            dd_mac(c, ah, al, x.h[i], x.l[i]);
            const DD d = dd_norm(c);
            y.h[i] = d.h;
            y.l[i] = d.l;
        }
    }
    __device__ static void xpay(Vec &y, const Vec &x, double b)
    {
        const float bh = (float)b, bl = (float)(b - (double)bh);
#pragma unroll
        for (int i = 0; i < 6; i++) {
            DAcc c = {x.h[i], x.l[i]};
            dd_mac(c, bh, bl, y.h[i], y.l[i]);
            const DD d = dd_norm(c);
            y.h[i] = d.h;
            y.l[i] = d.l;
        }
    }
    __device__ static void axpby(Vec &y, double a, const Vec &x, double b)
    {
        const float ah = (float)a, al = (float)(a - (double)ah);
        const float bh = (float)b, bl = (float)(b - (double)bh);
#pragma unroll
        for (int i = 0; i < 6; i++) {
            DAcc c = {0.f, 0.f};
            dd_mac(c, ah, al, x.h[i], x.l[i]);
            dd_mac(c, bh, bl, y.h[i], y.l[i]);
            const DD d = dd_norm(c);
            y.h[i] = d.h;
            y.l[i] = d.l;
        }
    }
    __device__ static double norm2(const Vec &x)
    {
        DAcc c = {0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 6; i++) dd_mac(c, x.h[i], x.l[i], x.h[i], x.l[i]);
        return (double)c.h + (double)c.e;
    }
    __device__ static void store(char *base, uint32_t s, const Vec &x)
    {
        float4 *q = reinterpret_cast<float4 *>(base + (size_t)s * T::SB);
        q[0] = make_float4(x.h[0], x.h[1], x.h[2], x.h[3]);
        q[1] = make_float4(x.h[4], x.h[5], x.l[0], x.l[1]);
        q[2] = make_float4(x.l[2], x.l[3], x.l[4], x.l[5]);
    }
    __device__ static double get(const Vec &x, int i) { return (double)x.h[i] + (double)x.l[i]; }
    __device__ static void set(Vec &x, int i, double d)
    {
        const float h = (float)d;
        x.h[i] = h;
        x.l[i] = (float)(d - (double)h);
    }
};

template <int P>
__device__ __forceinline__ void vload(const char *base, uint32_t s, typename Prec<P>::Vec &v)
{
    Prec<P>::load(base, s, v);
}

// ---------------------------------------------------------------- kernels
// r -= alpha Ap ; |r|^2 reduced with FIN_RR (beta, convergence flags)
template <int PS>
__global__ void __launch_bounds__(kVecBlock) k_update_r(VecRef r, VecRef Ap, Len len, Reduce red)
{
    const uint32_t Vh = len.n(blockIdx.y);
    using B = Blas<PS>;
    const int rhs = blockIdx.y;
    const double alpha = alpha_fresh_for_r(red.sc[rhs]) ? red.sc[rhs].alpha : 0.0;
    if constexpr (std::is_same<typename B::Vec, FloatArith::Vec>::value) {
        // FP32 records: the update and |r|^2 on the FP32 pipes, summed in float-float pairs
        // (per thread and per block), one FP64 conversion per block; this GPU issues FP64
        // operations at 1/64 of the FP32 rate, and an FP64 block sum in every thread of a
        // multi-right-hand-side grid costs more than the vector traffic
        FF acc[1] = {{0.f, 0.f}};
        if (alpha != 0.0) {
            const float af = (float)alpha;
            char *rp = r.rhs(rhs);
            const char *ap = Ap.rhs(rhs);
            for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
                typename B::Vec rv, av;
                vload<PS>(rp, s, rv);
                vload<PS>(ap, s, av);
                float n2 = 0.f;
#pragma unroll
                for (int i = 0; i < 6; i++) {
                    rv.v[i] = fmaf(-af, av.v[i], rv.v[i]);
                    n2 = fmaf(rv.v[i], rv.v[i], n2);
                }
                B::store(rp, s, rv);
                ff_add(acc[0], n2);
            }
        }
        block_sum_ff<1>(acc);
        double mine[1] = {threadIdx.x == 0 ? ff_value(acc[0]) : 0.0};
        grid_reduce<1>(red, mine, 1, rhs, gridDim.y, blockIdx.x);
        return;
    }
    double acc = 0.0;
    if (alpha != 0.0) {
        char *rp = r.rhs(rhs);
        const char *ap = Ap.rhs(rhs);
        for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
            typename B::Vec rv, av;
            vload<PS>(rp, s, rv);
            vload<PS>(ap, s, av);
            B::axpy(rv, -alpha, av);
            B::store(rp, s, rv);
            acc += B::norm2(rv);
        }
    }
    double mine[1] = {block_sum(acc)};
    grid_reduce<1>(red, mine, 1, rhs, gridDim.y, blockIdx.x);
}

// mode 0: x += alpha p, p = r + beta p;  mode 1: x += alpha p;  mode 2: p = r + beta p
template <int PS, int PX>
__global__ void __launch_bounds__(kVecBlock) k_update_xp(VecRef x, VecRef p, VecRef r, Len len, const Scalars *sc,
                                                         int mode, const LoopCtl *ctl)
{
    const uint32_t Vh = len.n(blockIdx.y);
    if (ctl) mode = ctl->mode; // inside a device-controlled loop
    using BS = Blas<PS>;
    using BX = Blas<PX>;
    const int rhs = blockIdx.y;
    const double alpha = alpha_fresh_for_x(sc[rhs]) ? sc[rhs].alpha : 0.0, beta = sc[rhs].beta;
    const bool do_x = mode != 2 && alpha != 0.0;
    const bool do_p = mode != 1 && sc[rhs].active;
    if (!do_x && !do_p) return;
    char *xp = x.rhs(rhs), *pp = p.rhs(rhs);
    const char *rp = r.rhs(rhs);
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
        typename BS::Vec pv;
        vload<PS>(pp, s, pv);
        if (do_x) {
            static_assert(std::is_same<typename BS::Vec, typename BX::Vec>::value, "shared vector type");
            typename BX::Vec xv;
            vload<PX>(xp, s, xv);
            BX::axpy(xv, alpha, pv);
            BX::store(xp, s, xv);
        }
        if (do_p) {
            typename BS::Vec rv;
            vload<PS>(rp, s, rv);
            BS::xpay(pv, rv, beta);
            BS::store(pp, s, pv);
        }
    }
}

// The update of a single-reduction CG iteration, after the Dslash epilogue's finishing step
// (FIN_AB) has produced alpha, beta and the flags of this iteration:
//   x += alpha p ; r -= alpha Ap ; p = r + beta p   (p only in mode 0 and while active)
// alpha is used only if it was produced by this iteration (astamp == it_all - 1).
template <int PS, int PX>
__global__ void __launch_bounds__(kVecBlock) k_update_xrp(VecRef x, VecRef p, VecRef r, VecRef Ap, Len len,
                                                          const Scalars *sc, int mode, const LoopCtl *ctl)
{
    const uint32_t Vh = len.n(blockIdx.y);
    if (ctl) mode = ctl->mode;
    using BS = Blas<PS>;
    using BX = Blas<PX>;
    static_assert(std::is_same<typename BS::Vec, typename BX::Vec>::value, "shared vector type");
    const int rhs = blockIdx.y;
    const Scalars &S = sc[rhs];
    const double alpha = alpha_fresh_for_x(S) ? S.alpha : 0.0, beta = S.beta;
    const bool do_xr = alpha != 0.0;
    const bool do_p = mode == 0 && S.active;
    if (!do_xr && !do_p) return;
    char *xp = x.rhs(rhs), *pp = p.rhs(rhs), *rp = r.rhs(rhs);
    const char *ap = Ap.rhs(rhs);
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
        typename BS::Vec pv, rv;
        vload<PS>(pp, s, pv);
        vload<PS>(rp, s, rv);
        if (do_xr) {
            typename BX::Vec xv;
            typename BS::Vec av;
            vload<PX>(xp, s, xv);
            vload<PS>(ap, s, av);
            BX::axpy(xv, alpha, pv);
            BS::axpy(rv, -alpha, av);
            BX::store(xp, s, xv);
            BS::store(rp, s, rv);
        }
        if (do_p) {
            BS::xpay(pv, rv, beta);
            BS::store(pp, s, pv);
        }
    }
}

// out (PB) = in (PA), element-wise through double components
template <int PA, int PB>
__global__ void __launch_bounds__(kVecBlock) k_convert(VecRef in, VecRef out, Len len)
{
    const uint32_t Vh = len.n(blockIdx.y);
    const int rhs = blockIdx.y;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
        typename Blas<PA>::Vec a;
        typename Blas<PB>::Vec b;
        vload<PA>(in.rhs(rhs), s, a);
#pragma unroll
        for (int i = 0; i < 6; i++) Blas<PB>::set(b, i, Blas<PA>::get(a, i));
        Blas<PB>::store(out.rhs(rhs), s, b);
    }
}

// x_hi (F64) += x_lo (PX); x_lo = 0
template <int PX>
__global__ void __launch_bounds__(kVecBlock) k_accum_hi(VecRef xhi, VecRef xlo, Len len)
{
    const uint32_t Vh = len.n(blockIdx.y);
    const int rhs = blockIdx.y;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
        typename Blas<PX>::Vec l, z;
        typename Blas<HISQ_F64>::Vec h;
        vload<PX>(xlo.rhs(rhs), s, l);
        vload<HISQ_F64>(xhi.rhs(rhs), s, h);
#pragma unroll
        for (int i = 0; i < 6; i++) {
            h.v[i] += Blas<PX>::get(l, i);
            Blas<PX>::set(z, i, 0.0);
        }
        Blas<HISQ_F64>::store(xhi.rhs(rhs), s, h);
        Blas<PX>::store(xlo.rhs(rhs), s, z);
    }
}

// r (F64) = b (F64) - Ax (PA) [- shift_rhs x (F64)]; |r|^2 reduced (FIN_STORE -> Scalars.last)
template <int PA>
__global__ void __launch_bounds__(kVecBlock) k_residual(VecRef b, VecRef Ax, VecRef r, Len len, Reduce red,
                                                        const double *shift = nullptr, VecRef x = VecRef{nullptr, 0})
{
    const uint32_t Vh = len.n(blockIdx.y);
    const int rhs = blockIdx.y;
    const double sh = shift ? shift[rhs] : 0.0;
    double acc = 0.0;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
        typename Blas<HISQ_F64>::Vec bv, rv, xv;
        typename Blas<PA>::Vec av;
        vload<HISQ_F64>(b.rhs(rhs), s, bv);
        vload<PA>(Ax.rhs(rhs), s, av);
        if (sh != 0.0) vload<HISQ_F64>(x.rhs(rhs), s, xv);
#pragma unroll
        for (int i = 0; i < 6; i++) {
            rv.v[i] = bv.v[i] - Blas<PA>::get(av, i);
            if (sh != 0.0) rv.v[i] -= sh * xv.v[i];
            acc = fma(rv.v[i], rv.v[i], acc);
        }
        Blas<HISQ_F64>::store(r.rhs(rhs), s, rv);
    }
    double mine[1] = {block_sum(acc)};
    grid_reduce<1>(red, mine, 1, rhs, gridDim.y, blockIdx.x);
}

// <a, b> = sum conj(a) b per right-hand side (complex), reduced with FIN_CDOT
template <int PV>
__global__ void __launch_bounds__(kVecBlock) k_cdot(VecRef a, VecRef b, Len len, Reduce red)
{
    const uint32_t Vh = len.n(blockIdx.y);
    const int rhs = blockIdx.y;
    if constexpr (std::is_same<typename Blas<PV>::Vec, FloatArith::Vec>::value) {
        // FP32 records: the site's products in FP32, float-float sums per thread and per
        // block, one FP64 conversion per block (FP64 issues at 1/64 of the FP32 rate here)
        FF d[2] = {{0.f, 0.f}, {0.f, 0.f}};
        for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
            typename Blas<PV>::Vec av, bv;
            vload<PV>(a.rhs(rhs), s, av);
            vload<PV>(b.rhs(rhs), s, bv);
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const float ar = av.v[2 * i], ai = av.v[2 * i + 1], br = bv.v[2 * i], bi = bv.v[2 * i + 1];
                sr = fmaf(ar, br, fmaf(ai, bi, sr));
                si = fmaf(ar, bi, fmaf(-ai, br, si));
            }
            ff_add(d[0], sr);
            ff_add(d[1], si);
        }
        block_sum_ff<2>(d);
        double mine[2] = {threadIdx.x == 0 ? ff_value(d[0]) : 0.0, threadIdx.x == 0 ? ff_value(d[1]) : 0.0};
        grid_reduce<2>(red, mine, 2, 2 * rhs, 2 * gridDim.y, blockIdx.x);
        return;
    }
    double re = 0.0, im = 0.0;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
        typename Blas<PV>::Vec av, bv;
        vload<PV>(a.rhs(rhs), s, av);
        vload<PV>(b.rhs(rhs), s, bv);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const double ar = Blas<PV>::get(av, 2 * i), ai = Blas<PV>::get(av, 2 * i + 1);
            const double br = Blas<PV>::get(bv, 2 * i), bi = Blas<PV>::get(bv, 2 * i + 1);
            re += ar * br + ai * bi;
            im += ar * bi - ai * br;
        }
    }
    double mine[2] = {block_sum(re), block_sum(im)};
    grid_reduce<2>(red, mine, 2, 2 * rhs, 2 * gridDim.y, blockIdx.x);
}

// After a reliable update replaced r: remove from p its component along r, then
// p = r + beta p, i.e. p = (1 - beta <r,p>/|r|^2) r + beta p  (complex coefficient)
template <int PV>
__global__ void __launch_bounds__(kVecBlock) k_p_reortho(VecRef p, VecRef r, Len len, const Scalars *sc)
{
    const uint32_t Vh = len.n(blockIdx.y);
    const int rhs = blockIdx.y;
    const Scalars &S = sc[rhs];
    if (!S.active) return;
    // the coefficients once per block (FP64 divisions in every thread of a large grid cost
    // more than the pass itself on this GPU's FP64 pipe)
    __shared__ double coef[3];
    if (threadIdx.x == 0) {
        const double beta = S.beta, rr = S.rr;
        coef[0] = rr > 0.0 ? 1.0 - beta * S.last / rr : 1.0;
        coef[1] = rr > 0.0 ? -beta * S.last_im / rr : 0.0;
        coef[2] = beta;
    }
    __syncthreads();
    const double cre = coef[0], cim = coef[1], beta = coef[2];
    if constexpr (std::is_same<typename Blas<PV>::Vec, FloatArith::Vec>::value) {
        // FP32 records: the coefficients converted once, the update in FP32
        const float cf = (float)cre, sf = (float)cim, bf = (float)beta;
        for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
            typename Blas<PV>::Vec pv, rv, out;
            vload<PV>(p.rhs(rhs), s, pv);
            vload<PV>(r.rhs(rhs), s, rv);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const float xr = rv.v[2 * i], xi = rv.v[2 * i + 1], yr = pv.v[2 * i], yi = pv.v[2 * i + 1];
                out.v[2 * i] = fmaf(cf, xr, fmaf(-sf, xi, bf * yr));
                out.v[2 * i + 1] = fmaf(cf, xi, fmaf(sf, xr, bf * yi));
            }
            Blas<PV>::store(p.rhs(rhs), s, out);
        }
        return;
    }
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
        typename Blas<PV>::Vec pv, rv, out;
        vload<PV>(p.rhs(rhs), s, pv);
        vload<PV>(r.rhs(rhs), s, rv);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const double xr = Blas<PV>::get(rv, 2 * i), xi = Blas<PV>::get(rv, 2 * i + 1);
            const double yr = Blas<PV>::get(pv, 2 * i), yi = Blas<PV>::get(pv, 2 * i + 1);
            Blas<PV>::set(out, 2 * i, cre * xr - cim * xi + beta * yr);
            Blas<PV>::set(out, 2 * i + 1, cre * xi + cim * xr + beta * yi);
        }
        Blas<PV>::store(p.rhs(rhs), s, out);
    }
}

// |x|^2 (F64) reduced with FIN_STORE
static __global__ void __launch_bounds__(kVecBlock) k_norm_f64(VecRef x, Len len, Reduce red)
{
    const uint32_t Vh = len.n(blockIdx.y);
    const int rhs = blockIdx.y;
    double acc = 0.0;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
        typename Blas<HISQ_F64>::Vec v;
        vload<HISQ_F64>(x.rhs(rhs), s, v);
#pragma unroll
        for (int i = 0; i < 6; i++) acc = fma(v.v[i], v.v[i], acc);
    }
    double mine[1] = {block_sum(acc)};
    grid_reduce<1>(red, mine, 1, rhs, gridDim.y, blockIdx.x);
}

}  // namespace hisq
