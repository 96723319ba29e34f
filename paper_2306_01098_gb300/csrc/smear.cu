// smear.cu -- HISQ fat and long links from thin links: two levels of smearing with a U(3)
// projection between them (Sec. 3.1).
//
// First level:  V = c1 U + c3 S3 + c5 S5 + c7 S7       (c1 1/8, c3 1/16, c5 1/64, c7 1/384)
// projection:   W = V (V^+ V)^(-1/2)                    (unitary polar factor of V)
// second level: X = c1 W + c3 S3 + c5 S5 + c7 S7 + cL L (c1 1, the same staples, cL -1/8)
// Naik:         N_mu(x) = cN W_mu(x) W_mu(x+mu) W_mu(x+2mu),   cN = -1/24 + eps/8
// with the staples of a field F_mu built from the links of the level (U, then W):
//   stap_nu[F]_mu(x) = U_nu(x) F_mu(x+nu) U_nu(x+mu)^+ + U_nu(x-nu)^+ F_mu(x-nu) U_nu(x-nu+mu)
//   S3 = sum_nu stap_nu[F];  S5 = sum_rho stap_rho[sum_{nu != rho} stap_nu[F]];
//   S7 = sum_sig stap_sig[sum_{rho != sig} stap_rho[sum_{nu != rho, sig} stap_nu[F]]];
//   L  = the staples whose detour is two steps along nu
// (all directions different from mu).  Everything is FP64.  One thread per (site, mu) builds
// every path on the fly; the set-up cost is paid once per gauge configuration.
// The projection uses the scaled Newton iteration for the polar decomposition,
//   X <- (g X + X^{-+} / g) / 2,  g = (|X^-1|_F / |X|_F)^(1/2)
// (N. J. Higham, "Computing the polar decomposition - with applications", SIAM J. Sci. Stat.
// Comput. 7 (1986)), which converges quadratically to the unitary factor.
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace hisq {
namespace smear {

struct M3 {
    double2 a[9];
};

__device__ __forceinline__ double2 cmul(double2 x, double2 y) { return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); }
__device__ __forceinline__ double2 cmulc(double2 x, double2 y) // x * conj(y)
{
    return make_double2(x.x * y.x + x.y * y.y, x.y * y.x - x.x * y.y);
}
__device__ __forceinline__ double2 ccmul(double2 x, double2 y) // conj(x) * y
{
    return make_double2(x.x * y.x + x.y * y.y, x.x * y.y - x.y * y.x);
}

__device__ __forceinline__ M3 zero()
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 9; i++) r.a[i] = make_double2(0.0, 0.0);
    return r;
}

// A B, A B^+, A^+ B
__device__ M3 mul(const M3 &A, const M3 &B)
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double2 s = make_double2(0.0, 0.0);
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const double2 p = cmul(A.a[3 * i + j], B.a[3 * j + k]);
                s.x += p.x;
                s.y += p.y;
            }
            r.a[3 * i + k] = s;
        }
    return r;
}
__device__ M3 mul_d(const M3 &A, const M3 &B)
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double2 s = make_double2(0.0, 0.0);
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const double2 p = cmulc(A.a[3 * i + j], B.a[3 * k + j]);
                s.x += p.x;
                s.y += p.y;
            }
            r.a[3 * i + k] = s;
        }
    return r;
}
__device__ M3 d_mul(const M3 &A, const M3 &B)
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double2 s = make_double2(0.0, 0.0);
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const double2 p = ccmul(A.a[3 * j + i], B.a[3 * j + k]);
                s.x += p.x;
                s.y += p.y;
            }
            r.a[3 * i + k] = s;
        }
    return r;
}
__device__ __forceinline__ void axpy(M3 &y, double c, const M3 &x)
{
#pragma unroll
    for (int i = 0; i < 9; i++) {
        y.a[i].x = fma(c, x.a[i].x, y.a[i].x);
        y.a[i].y = fma(c, x.a[i].y, y.a[i].y);
    }
}

struct Lat {
    int n[4];
    uint32_t V, Vh;
};

__device__ __forceinline__ uint32_t site_index(const Lat &L, const int (&c)[4])
{
    const uint32_t lex = (uint32_t)(c[0] + L.n[0] * (c[1] + L.n[1] * (c[2] + L.n[2] * c[3])));
    return (lex >> 1) + L.Vh * (uint32_t)((c[0] + c[1] + c[2] + c[3]) & 1);
}

// the link of direction mu at the site c + k * hat(d) (periodic)
__device__ __forceinline__ M3 load(const Lat &L, const double2 *f, int mu, const int (&c)[4], int d = 0, int k = 0,
                                   int d2 = 0, int k2 = 0)
{
    int y[4] = {c[0], c[1], c[2], c[3]};
    y[d] = ((y[d] + k) % L.n[d] + L.n[d]) % L.n[d];
    y[d2] = ((y[d2] + k2) % L.n[d2] + L.n[d2]) % L.n[d2];
    const double2 *p = f + ((size_t)mu * L.V + site_index(L, y)) * 9;
    M3 r;
#pragma unroll
    for (int i = 0; i < 9; i++) r.a[i] = __ldg(p + i);
    return r;
}

__device__ __forceinline__ void move(const Lat &L, int (&y)[4], int d, int k)
{
    y[d] = ((y[d] + k) % L.n[d] + L.n[d]) % L.n[d];
}

// stap_nu[F]_mu(y), F = the field f of direction mu, links u
__device__ M3 stap1(const Lat &L, const double2 *u, const double2 *f, int mu, int nu, const int (&y)[4])
{
    // U_nu(y) F(y+nu) U_nu(y+mu)^+
    M3 r = mul_d(mul(load(L, u, nu, y), load(L, f, mu, y, nu, 1)), load(L, u, nu, y, mu, 1));
    // U_nu(y-nu)^+ F(y-nu) U_nu(y-nu+mu)
    const M3 b = mul(d_mul(load(L, u, nu, y, nu, -1), load(L, f, mu, y, nu, -1)), load(L, u, nu, y, nu, -1, mu, 1));
    axpy(r, 1.0, b);
    return r;
}

// stap_rho[stap_nu[F]]_mu(y)
__device__ M3 stap2(const Lat &L, const double2 *u, const double2 *f, int mu, int rho, int nu, const int (&y)[4])
{
    int yp[4] = {y[0], y[1], y[2], y[3]}, ym[4] = {y[0], y[1], y[2], y[3]};
    move(L, yp, rho, 1);
    move(L, ym, rho, -1);
    M3 r = mul_d(mul(load(L, u, rho, y), stap1(L, u, f, mu, nu, yp)), load(L, u, rho, y, mu, 1));
    const M3 b = mul(d_mul(load(L, u, rho, y, rho, -1), stap1(L, u, f, mu, nu, ym)), load(L, u, rho, ym, mu, 1));
    axpy(r, 1.0, b);
    return r;
}

// stap_sig[stap_rho[stap_nu[F]]]_mu(y)
__device__ M3 stap3(const Lat &L, const double2 *u, const double2 *f, int mu, int sig, int rho, int nu, const int (&y)[4])
{
    int yp[4] = {y[0], y[1], y[2], y[3]}, ym[4] = {y[0], y[1], y[2], y[3]};
    move(L, yp, sig, 1);
    move(L, ym, sig, -1);
    M3 r = mul_d(mul(load(L, u, sig, y), stap2(L, u, f, mu, rho, nu, yp)), load(L, u, sig, y, mu, 1));
    const M3 b = mul(d_mul(load(L, u, sig, y, sig, -1), stap2(L, u, f, mu, rho, nu, ym)), load(L, u, sig, ym, mu, 1));
    axpy(r, 1.0, b);
    return r;
}

// the staple whose detour is two steps along nu
__device__ M3 lepage(const Lat &L, const double2 *u, const double2 *f, int mu, int nu, const int (&y)[4])
{
    // U_nu(y) U_nu(y+nu) F(y+2nu) [U_nu(y+mu) U_nu(y+mu+nu)]^+
    const M3 up = mul(load(L, u, nu, y), load(L, u, nu, y, nu, 1));
    const M3 upm = mul(load(L, u, nu, y, mu, 1), load(L, u, nu, y, mu, 1, nu, 1));
    M3 r = mul_d(mul(up, load(L, f, mu, y, nu, 2)), upm);
    // [U_nu(y-2nu) U_nu(y-nu)]^+ F(y-2nu) U_nu(y-2nu+mu) U_nu(y-nu+mu)
    const M3 dn = mul(load(L, u, nu, y, nu, -2), load(L, u, nu, y, nu, -1));
    const M3 dnm = mul(load(L, u, nu, y, nu, -2, mu, 1), load(L, u, nu, y, nu, -1, mu, 1));
    axpy(r, 1.0, mul(d_mul(dn, load(L, f, mu, y, nu, -2)), dnm));
    return r;
}

struct Coef {
    double c1, c3, c5, c7, cl;
};

// out_mu(x) = c1 F + c3 S3 + c5 S5 + c7 S7 + cl L, one thread per (site, mu)
__global__ void __launch_bounds__(64) k_smear_level(Lat L, const double2 *u, const double2 *f, double2 *out, Coef c)
{
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= 4ull * L.V) return;
    const int mu = (int)(t / L.V);
    uint32_t lex = (uint32_t)(t - (uint64_t)mu * L.V);
    int x[4];
#pragma unroll
    for (int d = 0; d < 4; d++) {
        x[d] = (int)(lex % (uint32_t)L.n[d]);
        lex /= (uint32_t)L.n[d];
    }
    M3 acc = zero();
    axpy(acc, c.c1, load(L, f, mu, x));
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        axpy(acc, c.c3, stap1(L, u, f, mu, nu, x));
        if (c.cl != 0.0) axpy(acc, c.cl, lepage(L, u, f, mu, nu, x));
    }
    for (int rho = 0; rho < 4; rho++) {
        if (rho == mu) continue;
        for (int nu = 0; nu < 4; nu++) {
            if (nu == mu || nu == rho) continue;
            axpy(acc, c.c5, stap2(L, u, f, mu, rho, nu, x));
        }
    }
    for (int sig = 0; sig < 4; sig++) {
        if (sig == mu) continue;
        for (int rho = 0; rho < 4; rho++) {
            if (rho == mu || rho == sig) continue;
            for (int nu = 0; nu < 4; nu++) {
                if (nu == mu || nu == rho || nu == sig) continue;
                axpy(acc, c.c7, stap3(L, u, f, mu, sig, rho, nu, x));
            }
        }
    }
    double2 *p = out + ((size_t)mu * L.V + site_index(L, x)) * 9;
#pragma unroll
    for (int i = 0; i < 9; i++) p[i] = acc.a[i];
}

// inverse of a 3x3 complex matrix by cofactors; returns false if singular
__device__ bool inverse(const M3 &A, M3 &inv)
{
    const double2 *a = A.a;
    double2 cof[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            const double2 p = cmul(a[3 * i1 + j1], a[3 * i2 + j2]), q = cmul(a[3 * i1 + j2], a[3 * i2 + j1]);
            cof[3 * i + j] = make_double2(p.x - q.x, p.y - q.y);
        }
    double2 det = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const double2 p = cmul(a[j], cof[j]);
        det.x += p.x;
        det.y += p.y;
    }
    const double dd = det.x * det.x + det.y * det.y;
    if (!(dd > 0.0) || !isfinite(dd)) return false;
    const double2 rdet = make_double2(det.x / dd, -det.y / dd);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) inv.a[3 * i + j] = cmul(cof[3 * j + i], rdet); // adjugate / det
    return true;
}

__device__ __forceinline__ double fro2(const M3 &A)
{
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 9; i++) s += A.a[i].x * A.a[i].x + A.a[i].y * A.a[i].y;
    return s;
}

// W = unitary polar factor of V (scaled Newton iteration); a singular or non-converging
// matrix raises the device error flag
__global__ void __launch_bounds__(128) k_project_u3(const double2 *v, double2 *w, uint64_t n, DevStatus *status)
{
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    M3 X;
#pragma unroll
    for (int i = 0; i < 9; i++) X.a[i] = v[t * 9 + i];
    bool ok = false;
    for (int it = 0; it < 30; it++) {
        M3 Xi;
        if (!inverse(X, Xi)) break;
        const double g = sqrt(sqrt(fro2(Xi) / fro2(X)));
        M3 Y;
        double diff = 0.0;
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                // (X^-1)^+ = conj of the transposed inverse
                const double2 xi = Xi.a[3 * c + r];
                const double2 y = make_double2(0.5 * (g * X.a[3 * r + c].x + xi.x / g),
                                               0.5 * (g * X.a[3 * r + c].y - xi.y / g));
                const double dx = y.x - X.a[3 * r + c].x, dy = y.y - X.a[3 * r + c].y;
                diff += dx * dx + dy * dy;
                Y.a[3 * r + c] = y;
            }
        X = Y;
        // quadratic convergence: a change of 1e-12 leaves an error of order 1e-24
        if (diff <= 1e-24 * fro2(X)) {
            ok = true;
            break;
        }
    }
#pragma unroll
    for (int i = 0; i < 9; i++) w[t * 9 + i] = X.a[i];
    if (!ok && status) {
        status->where = 2; // link projection
        atomicExch(&status->error, (int)HISQ_EDEVICE);
    }
}

// N_mu(x) = cN W_mu(x) W_mu(x+mu) W_mu(x+2mu)
__global__ void __launch_bounds__(128) k_naik(Lat L, const double2 *w, double2 *out, double cn)
{
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= 4ull * L.V) return;
    const int mu = (int)(t / L.V);
    uint32_t lex = (uint32_t)(t - (uint64_t)mu * L.V);
    int x[4];
#pragma unroll
    for (int d = 0; d < 4; d++) {
        x[d] = (int)(lex % (uint32_t)L.n[d]);
        lex /= (uint32_t)L.n[d];
    }
    const M3 r = mul(mul(load(L, w, mu, x), load(L, w, mu, x, mu, 1)), load(L, w, mu, x, mu, 2));
    double2 *p = out + ((size_t)mu * L.V + site_index(L, x)) * 9;
#pragma unroll
    for (int i = 0; i < 9; i++) p[i] = make_double2(cn * r.a[i].x, cn * r.a[i].y);
}

}  // namespace smear
}  // namespace hisq

using namespace hisq;

extern "C" int hisq_smear_links(const int dims[4], const double *thin, double *fat, double *lng, double eps_naik,
                                int links_on_device, void *stream)
{
    if (!dims || !thin || !fat || !lng || !std::isfinite(eps_naik)) return HISQ_EINVAL;
    smear::Lat L{};
    uint64_t V = 1;
    for (int d = 0; d < 4; d++) {
        if (dims[d] < 4 || dims[d] % 2) return HISQ_EINVAL;
        L.n[d] = dims[d];
        V *= (uint64_t)dims[d];
    }
    if (V > (1ull << 31)) return HISQ_EINVAL;
    L.V = (uint32_t)V;
    L.Vh = (uint32_t)(V / 2);
    const size_t bytes = 4 * V * 9 * sizeof(double2);
    cudaStream_t st = (cudaStream_t)stream;
    double2 *u = nullptr, *v = nullptr, *w = nullptr, *x = nullptr, *nk = nullptr;
    DevStatus *status = nullptr;
    auto release = [&]() {
        for (void *p : {(void *)u, (void *)v, (void *)w, (void *)x, (void *)nk, (void *)status})
            if (p) cudaFree(p);
    };
    bool ok = cudaMalloc((void **)&u, bytes) == cudaSuccess && cudaMalloc((void **)&v, bytes) == cudaSuccess &&
              cudaMalloc((void **)&w, bytes) == cudaSuccess && cudaMalloc((void **)&status, sizeof(DevStatus)) == cudaSuccess;
    if (ok && !links_on_device) ok = cudaMalloc((void **)&x, bytes) == cudaSuccess && cudaMalloc((void **)&nk, bytes) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release();
        return HISQ_ENOMEM;
    }
    double2 *xo = links_on_device ? reinterpret_cast<double2 *>(fat) : x;
    double2 *no = links_on_device ? reinterpret_cast<double2 *>(lng) : nk;
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(DevStatus), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(u, thin, bytes, links_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    const unsigned nb64 = (unsigned)((4 * V + 63) / 64), nb128 = (unsigned)((4 * V + 127) / 128);
    if (e == cudaSuccess) {
        smear::k_smear_level<<<nb64, 64, 0, st>>>(L, u, u, v, smear::Coef{1.0 / 8, 1.0 / 16, 1.0 / 64, 1.0 / 384, 0.0});
        smear::k_project_u3<<<nb128, 128, 0, st>>>(v, w, 4 * V, status);
        smear::k_smear_level<<<nb64, 64, 0, st>>>(L, w, w, xo, smear::Coef{1.0, 1.0 / 16, 1.0 / 64, 1.0 / 384, -1.0 / 8});
        smear::k_naik<<<nb128, 128, 0, st>>>(L, w, no, -1.0 / 24 + eps_naik / 8);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !links_on_device) {
        e = cudaMemcpyAsync(fat, xo, bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lng, no, bytes, cudaMemcpyDeviceToHost, st);
    }
    DevStatus h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? HISQ_ENOMEM : HISQ_ECUDA;
    }
    return h.error ? HISQ_EDEVICE : HISQ_OK;
}
