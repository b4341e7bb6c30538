// Network-parameter extraction on the GPU in FP64 (Sec. II-A of arXiv 2208.04371):
//   Z_r (Eq. 2), power-mode S* (Eq. 1), renormalisation to z_ref (Eq. 5-6), the overall
//   characteristic impedance from the ABCD matrix of S*, and the phase delay (Eq. 8).
// One thread per frequency for the matrix work, one thread per (i, j) pair for the
// unwrapped phase (a sequential scan over increasing frequency).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "yf_grid.h"
#include "yf_internal.h"

namespace yf {
namespace {

constexpr int kMaxN = 8;

struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx mk(double r, double i) { return {r, i}; }
__device__ __forceinline__ cplx add(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx sub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx mul(cplx a, cplx b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cplx dvd(cplx a, cplx b)
{
    // Smith's algorithm
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, den = b.re + b.im * r;
        return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
    }
    const double r = b.re / b.im, den = b.re * r + b.im;
    return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
}
__device__ __forceinline__ double cabs_(cplx a) { return hypot(a.re, a.im); }
// principal square root; both radicands are clamped at zero, because |z| rounded by hypot
// can fall an ulp below |Re z| for an (almost) real argument
__device__ __forceinline__ cplx csqrt_(cplx z)
{
    const double r = cabs_(z);
    const double a = sqrt(0.5 * fmax(r + z.re, 0.0));
    const double b = sqrt(0.5 * fmax(r - z.re, 0.0));
    return {a, z.im < 0 ? -b : b};
}

// in-place inverse of an n x n complex matrix (Gauss-Jordan, partial pivoting)
__device__ bool inverse(cplx *A, cplx *Ai, int n)
{
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ai[r * n + c] = mk(r == c ? 1.0 : 0.0, 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = cabs_(A[c * n + c]);
        for (int r = c + 1; r < n; ++r)
            if (cabs_(A[r * n + c]) > best) { best = cabs_(A[r * n + c]); piv = r; }
        if (best == 0.0) return false;
        if (piv != c)
            for (int q = 0; q < n; ++q) {
                cplx t = A[c * n + q]; A[c * n + q] = A[piv * n + q]; A[piv * n + q] = t;
                t = Ai[c * n + q]; Ai[c * n + q] = Ai[piv * n + q]; Ai[piv * n + q] = t;
            }
        const cplx d = A[c * n + c];
        for (int q = 0; q < n; ++q) {
            A[c * n + q] = dvd(A[c * n + q], d);
            Ai[c * n + q] = dvd(Ai[c * n + q], d);
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const cplx f = A[r * n + c];
            for (int q = 0; q < n; ++q) {
                A[r * n + q] = sub(A[r * n + q], mul(f, A[c * n + q]));
                Ai[r * n + q] = sub(Ai[r * n + q], mul(f, Ai[c * n + q]));
            }
        }
    }
    return true;
}

struct SpArgs {
    int n, nf, uniform, dir1;
    double z_ref;
    // inputs, complex [..][nf]: Vinc[j], Iinc[j], Vtot[j*n + i]
    const cplx *vinc, *iinc, *vtot;
    // outputs (device)
    cplx *sstar, *s, *zr, *zc;
};

__global__ void k_sparams(SpArgs A)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= A.nf) return;
    const int n = A.n;
    cplx Zr[kMaxN], Ss[kMaxN * kMaxN];
    if (A.uniform) {
        // one run driven at port 0 of a uniform two-port: the forward wave crosses port 1
        // against its own incident direction
        const cplx v0 = A.vinc[f], i0 = A.iinc[f], v1 = A.vinc[A.nf + f], i1 = A.iinc[A.nf + f];
        Zr[0] = dvd(v0, i0);
        Zr[1] = dvd(v1, mk(A.dir1 * i1.re, A.dir1 * i1.im));
        const cplx s21 = mul(dvd(v1, v0), csqrt_(dvd(Zr[0], Zr[1])));
        Ss[0] = mk(0, 0); Ss[3] = mk(0, 0); Ss[1] = s21; Ss[2] = s21;
    } else {
        for (int j = 0; j < n; ++j) Zr[j] = dvd(A.vinc[j * A.nf + f], A.iinc[j * A.nf + f]);   // Eq. 2
        for (int j = 0; j < n; ++j) {
            const cplx vi = A.vinc[j * A.nf + f];
            for (int i = 0; i < n; ++i) {
                const cplx vt = A.vtot[(j * n + i) * A.nf + f];
                if (i == j) Ss[j * n + j] = dvd(sub(vt, vi), vi);                              // Eq. 1, i = j
                else Ss[i * n + j] = mul(dvd(vt, vi), csqrt_(dvd(Zr[j], Zr[i])));              // Eq. 1, i != j
            }
        }
    }
    for (int q = 0; q < n * n; ++q) A.sstar[(size_t)f * n * n + q] = Ss[q];
    for (int i = 0; i < n; ++i) A.zr[(size_t)i * A.nf + f] = Zr[i];

    // Eq. 5-6: S = A^{-1} (S* - B)(I - B S*)^{-1} A, B = diag((z - Zr)/(z + Zr)),
    // A = G*^{-1} G (I - B), G = diag(1/sqrt|Re Zr|), G* = 1/sqrt(z)
    cplx B[kMaxN], Ad[kMaxN];
    const cplx z = mk(A.z_ref, 0.0);
    for (int i = 0; i < n; ++i) {
        B[i] = dvd(sub(z, Zr[i]), add(z, Zr[i]));
        const double gs = sqrt(A.z_ref) / sqrt(fabs(Zr[i].re));
        const cplx omb = sub(mk(1, 0), B[i]);
        Ad[i] = mk(gs * omb.re, gs * omb.im);
    }
    cplx T[kMaxN * kMaxN], Ti[kMaxN * kMaxN];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            const cplx bs = mul(B[r], Ss[r * n + c]);
            T[r * n + c] = sub(mk(r == c ? 1.0 : 0.0, 0.0), bs);
        }
    const bool ok = inverse(T, Ti, n);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            cplx m = mk(0, 0);
            for (int q = 0; q < n; ++q) {
                const cplx lhs = (r == q) ? sub(Ss[r * n + q], B[r]) : Ss[r * n + q];
                m = add(m, mul(lhs, Ti[q * n + c]));
            }
            const cplx v = ok ? mul(dvd(m, Ad[r]), Ad[c]) : mk(NAN, NAN);
            A.s[(size_t)f * n * n + r * n + c] = v;
        }

    // overall characteristic impedance (two-port): Z = R (I + S*)(I - S*)^{-1} R,
    // R = diag(sqrt(Zr)); ABCD: B = det Z / Z21, C = 1 / Z21; Zc = sqrt(B / C), Re >= 0
    if (n == 2 && A.zc) {
        cplx P[4], Pi[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) P[r * 2 + c] = sub(mk(r == c ? 1.0 : 0.0, 0.0), Ss[r * 2 + c]);
        cplx zc = mk(NAN, NAN);
        if (inverse(P, Pi, 2)) {
            cplx Zm[4];
            const cplx R[2] = {csqrt_(Zr[0]), csqrt_(Zr[1])};
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) {
                    cplx m = mk(0, 0);
                    for (int q = 0; q < 2; ++q) {
                        const cplx ip = add(mk(r == q ? 1.0 : 0.0, 0.0), Ss[r * 2 + q]);
                        m = add(m, mul(ip, Pi[q * 2 + c]));
                    }
                    Zm[r * 2 + c] = mul(mul(R[r], m), R[c]);
                }
            const cplx det = sub(mul(Zm[0], Zm[3]), mul(Zm[1], Zm[2]));
            const cplx Bm = dvd(det, Zm[2]);
            const cplx Cm = dvd(mk(1, 0), Zm[2]);
            zc = csqrt_(dvd(Bm, Cm));
            if (zc.re < 0) zc = mk(-zc.re, -zc.im);
        }
        A.zc[f] = zc;
    }
}

// Eq. 8: tau = theta / (360 f), theta = -unwrap(arg S*_ij) in degrees
__global__ void k_phase_delay(const cplx *sstar, const double *freqs, int n, int nf, double *tau)
{
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= n * n) return;
    const int i = pr / n, j = pr % n;
    double prev = 0.0, offset = 0.0;
    for (int f = 0; f < nf; ++f) {
        double t = 0.0;
        if (i != j) {
            const cplx s = sstar[(size_t)f * n * n + i * n + j];
            const double ph = atan2(s.im, s.re) * (180.0 / 3.14159265358979323846);
            if (f > 0) {
                const double d = ph - prev;
                if (d > 180.0) offset -= 360.0;
                else if (d < -180.0) offset += 360.0;
            }
            prev = ph;
            t = -(ph + offset) / (360.0 * freqs[f]);
        }
        tau[(size_t)f * n * n + i * n + j] = t;
    }
}

// principal complex logarithm and inverse hyperbolic cosine, acosh z = log(z + sqrt(z+1) sqrt(z-1))
__device__ __forceinline__ cplx clog_(cplx z) { return {log(cabs_(z)), atan2(z.im, z.re)}; }
__device__ __forceinline__ cplx cacosh_(cplx z)
{
    return clog_(add(z, mul(csqrt_(add(z, mk(1, 0))), csqrt_(sub(z, mk(1, 0))))));
}

// Telegrapher's model of a two-port (end of Sec. II-A): S* -> Z (pseudo-waves with the port
// references) -> ABCD; gamma l = +-acosh((A + D)/2) + 2 pi j k (cosh is even and periodic).
// acosh folds beta l into [0, pi], so one thread walks the frequencies in order: the lowest
// takes beta l in [0, pi], every further one the candidate nearest beta l grown in proportion
// to f from the last frequency with a finite result; alpha's sign follows from beta > 0.
// Z_c = sqrt(B/C) with Re >= 0; R + j w L = gamma Z_c, G + j w C = gamma / Z_c per unit length.
// A singular conversion (I - S* not invertible) gives NaN at that frequency only.
__global__ void k_rlcg(const cplx *sstar, const cplx *zr, const double *freqs, int nf, double length,
                       cplx *gamma, double *R, double *L, double *G, double *C)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const double twopi = 6.283185307179586476925286766559;
    cplx prev = mk(0, 0);
    double fprev = 0.0;
    bool have = false;
    for (int f = 0; f < nf; ++f) {
        cplx S[4], P[4], Pi[4];
        for (int q = 0; q < 4; ++q) S[q] = sstar[(size_t)f * 4 + q];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) P[r * 2 + c] = sub(mk(r == c ? 1.0 : 0.0, 0.0), S[r * 2 + c]);
        cplx g = mk(NAN, NAN), zc = mk(NAN, NAN);
        if (inverse(P, Pi, 2)) {
            const cplx rt[2] = {csqrt_(zr[f]), csqrt_(zr[nf + f])};
            cplx Z[4];
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) {
                    cplx m = mk(0, 0);
                    for (int q = 0; q < 2; ++q)
                        m = add(m, mul(add(mk(r == q ? 1.0 : 0.0, 0.0), S[r * 2 + q]), Pi[q * 2 + c]));
                    Z[r * 2 + c] = mul(mul(rt[r], m), rt[c]);
                }
            const cplx A = dvd(Z[0], Z[2]), D = dvd(Z[3], Z[2]);
            const cplx Bm = dvd(sub(mul(Z[0], Z[3]), mul(Z[1], Z[2])), Z[2]);
            const cplx Cm = dvd(mk(1, 0), Z[2]);
            zc = csqrt_(dvd(Bm, Cm));
            if (zc.re < 0) zc = mk(-zc.re, -zc.im);
            g = cacosh_(mk(0.5 * (A.re + D.re), 0.5 * (A.im + D.im)));
        }
        const bool finite = isfinite(g.re) && isfinite(g.im) && isfinite(zc.re) && isfinite(zc.im);
        if (finite) {
            if (!have) {
                if (!(g.im > 0 || (g.im == 0 && g.re >= 0))) g = mk(-g.re, -g.im);
            } else {
                const double pred = prev.im * freqs[f] / fprev;
                const cplx cand[2] = {g, mk(-g.re, -g.im)};
                for (int q = 0; q < 2; ++q) {
                    const cplx c = cand[q];
                    const cplx cs = mk(c.re, c.im + twopi * rint((pred - c.im) / twopi));
                    if (q == 0 || fabs(cs.im - pred) < fabs(g.im - pred)) g = cs;
                }
            }
            prev = g;
            fprev = freqs[f];
            have = true;
        } else {
            g = mk(NAN, NAN);
            zc = mk(NAN, NAN);
        }
        const cplx gam = mk(g.re / length, g.im / length);
        const cplx zs = mul(gam, zc), yp = dvd(gam, zc);
        const double w = twopi * freqs[f];
        if (gamma) gamma[f] = gam;
        R[f] = zs.re;
        L[f] = zs.im / w;
        G[f] = yp.re;
        C[f] = yp.im / w;
    }
}

yf_status run_sparams(int n, int nf, const double *freqs, const std::vector<double> &vinc,
                      const std::vector<double> &iinc, const std::vector<double> &vtot, int uniform,
                      int dir1, double z_ref, double *S_star, double *S, double *Zr, double *Zc,
                      double *tau)
{
    const size_t nn = (size_t)n * n;
    // one device block: inputs, outputs, freqs
    const size_t n_in = vinc.size() + iinc.size() + vtot.size();
    const size_t n_out = 2 * nf * nn * 2 + 2 * (size_t)n * nf + 2 * (size_t)nf + nf * nn;
    double *buf = nullptr;
    YF_CUDA_TRY(cudaMalloc(&buf, (n_in + n_out + nf) * sizeof(double)));
    std::vector<double> host(n_in + nf);
    size_t o = 0;
    for (double v : vinc) host[o++] = v;
    for (double v : iinc) host[o++] = v;
    for (double v : vtot) host[o++] = v;
    for (int f = 0; f < nf; ++f) host[o++] = freqs[f];
    cudaError_t e = cudaMemcpy(buf, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(buf); return cuda_fail(e, "sparams upload"); }
    SpArgs A;
    A.n = n; A.nf = nf; A.uniform = uniform; A.dir1 = dir1; A.z_ref = z_ref;
    A.vinc = (const cplx *)buf;
    A.iinc = (const cplx *)(buf + vinc.size());
    A.vtot = (const cplx *)(buf + vinc.size() + iinc.size());
    const double *fr = buf + n_in;
    double *out = buf + n_in + nf;
    A.sstar = (cplx *)out;
    A.s = (cplx *)(out + 2 * nf * nn);
    A.zr = (cplx *)(out + 4 * nf * nn);
    A.zc = (cplx *)(out + 4 * nf * nn + 2 * (size_t)n * nf);
    double *tau_d = out + 4 * nf * nn + 2 * (size_t)n * nf + 2 * (size_t)nf;
    k_sparams<<<(nf + 63) / 64, 64>>>(A);
    k_phase_delay<<<1, 64>>>(A.sstar, fr, n, nf, tau_d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    std::vector<double> res(n_out);
    if (e == cudaSuccess) e = cudaMemcpy(res.data(), out, n_out * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "sparams kernel");
    const double *r = res.data();
    if (S_star) for (size_t q = 0; q < 2 * nf * nn; ++q) S_star[q] = r[q];
    if (S) for (size_t q = 0; q < 2 * nf * nn; ++q) S[q] = r[2 * nf * nn + q];
    if (Zr) for (size_t q = 0; q < 2 * (size_t)n * nf; ++q) Zr[q] = r[4 * nf * nn + q];
    if (Zc && n == 2) for (size_t q = 0; q < 2 * (size_t)nf; ++q) Zc[q] = r[4 * nf * nn + 2 * n * nf + q];
    if (tau) for (size_t q = 0; q < nf * nn; ++q) tau[q] = r[4 * nf * nn + 2 * n * nf + 2 * nf + q];
    return YF_OK;
}

}  // namespace

yf_status sparams_uniform(int nf, const double *freqs, const double *d, int dir1, double z_ref,
                          double *S_star, double *S, double *Zr, double *Zc, double *tau)
{
    // d: [port][Vre, Vim, Ire, Iim][nf] -> complex interleaved per port
    std::vector<double> vinc(4 * (size_t)nf), iinc(4 * (size_t)nf), vtot;
    for (int p = 0; p < 2; ++p)
        for (int f = 0; f < nf; ++f) {
            vinc[2 * (p * nf + f)] = d[(4 * p + 0) * nf + f];
            vinc[2 * (p * nf + f) + 1] = d[(4 * p + 1) * nf + f];
            iinc[2 * (p * nf + f)] = d[(4 * p + 2) * nf + f];
            iinc[2 * (p * nf + f) + 1] = d[(4 * p + 3) * nf + f];
        }
    return run_sparams(2, nf, freqs, vinc, iinc, vtot, 1, dir1, z_ref, S_star, S, Zr, Zc, tau);
}

}  // namespace yf

extern "C" yf_status yf_sparams(int nports, int nfreq, const double *freqs, const yf_port_dfts *inc,
                                const yf_port_dfts *tot, double z_ref, double *S_star, double *S,
                                double *Zr, double *Zc, double *tau)
{
    using namespace yf;
    if (nports < 1 || nports > kMaxN || nfreq < 1 || !freqs || !inc || !tot || !(z_ref > 0))
        return fail(YF_E_INVALID, "yf_sparams: bad arguments (1 <= nports <= %d)", kMaxN);
    const int n = nports, nf = nfreq;
    std::vector<double> vinc(2 * (size_t)n * nf), iinc(2 * (size_t)n * nf), vtot(2 * (size_t)n * n * nf);
    for (int j = 0; j < n; ++j) {
        const yf_port_dfts &a = inc[j];
        if (!a.V_re || !a.V_im || !a.I_re || !a.I_im) return fail(YF_E_INVALID, "yf_sparams: NULL spectrum");
        for (int f = 0; f < nf; ++f) {
            vinc[2 * (j * nf + f)] = a.V_re[f]; vinc[2 * (j * nf + f) + 1] = a.V_im[f];
            iinc[2 * (j * nf + f)] = a.I_re[f]; iinc[2 * (j * nf + f) + 1] = a.I_im[f];
        }
        for (int i = 0; i < n; ++i) {
            const yf_port_dfts &t = tot[j * n + i];
            if (!t.V_re || !t.V_im) return fail(YF_E_INVALID, "yf_sparams: NULL spectrum");
            for (int f = 0; f < nf; ++f) {
                vtot[2 * ((j * n + i) * nf + f)] = t.V_re[f];
                vtot[2 * ((j * n + i) * nf + f) + 1] = t.V_im[f];
            }
        }
    }
    return run_sparams(n, nf, freqs, vinc, iinc, vtot, 0, 1, z_ref, S_star, S, Zr, Zc, tau);
}

extern "C" yf_status yf_rlcg(int nfreq, const double *freqs, const double *S_star, const double *Zr,
                             double length, double *gamma, double *R, double *L, double *G, double *C)
{
    using namespace yf;
    if (nfreq < 1 || !freqs || !S_star || !Zr || !R || !L || !G || !C || !(length > 0))
        return fail(YF_E_INVALID, "yf_rlcg: bad arguments");
    for (int f = 0; f < nfreq; ++f)
        if (!(freqs[f] > 0) || (f > 0 && !(freqs[f] > freqs[f - 1])))
            return fail(YF_E_INVALID, "yf_rlcg: frequencies must be positive and increasing");
    const int nf = nfreq;
    // device staging: S* [F][4], Zr [2][F] (complex), freqs [F], outputs gamma [F] + 4 x [F]
    const size_t in_c = (size_t)6 * nf, out_d = (size_t)2 * nf + 4 * (size_t)nf;
    double *buf = nullptr;
    YF_CUDA_TRY(cudaMalloc(&buf, (2 * in_c + nf + out_d) * sizeof(double)));
    cplx *ds = (cplx *)buf, *dz = ds + 4 * nf;
    double *dfq = buf + 2 * in_c, *dout = dfq + nf;
    cudaError_t e = cudaMemcpy(ds, S_star, (size_t)4 * nf * sizeof(cplx), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dz, Zr, (size_t)2 * nf * sizeof(cplx), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dfq, freqs, nf * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_rlcg<<<1, 1>>>(ds, dz, dfq, nf, length, (cplx *)dout, dout + 2 * nf, dout + 3 * nf,
                         dout + 4 * nf, dout + 5 * nf);
        e = cudaGetLastError();
    }
    std::vector<double> h(out_d);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), dout, out_d * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "yf_rlcg");
    if (gamma) for (size_t q = 0; q < 2 * (size_t)nf; ++q) gamma[q] = h[q];
    for (int f = 0; f < nf; ++f) {
        R[f] = h[2 * nf + f];
        L[f] = h[3 * nf + f];
        G[f] = h[4 * nf + f];
        C[f] = h[5 * nf + f];
    }
    return YF_OK;
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant of the extraction above.  Its only scratch, the power-mode
// matrix S* that the phase-delay pass reads back, lives in a fixed device array instead of
// a per-call cudaMalloc, and the caller provides every input and output on the device.

#include <cudaTypedefs.h>
#include <mutex>

namespace yf {
namespace {

constexpr int kNoAllocMaxEntries = 32768;   // nfreq * nports^2 complex entries (512 KiB)
constexpr int kNoAllocMaxDevices = 64;

// One copy per GPU that loads this library, kept until the process exits.  Host code must
// not pass the symbol itself to a kernel: on the host it names a stand-in, not device
// memory.  The device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) cplx g_noalloc_sstar[kNoAllocMaxEntries];

// The device address of the array as last looked up on each device, with the context it
// was looked up in: a context that is destroyed and created again (cudaDeviceReset) loads
// the module afresh, and the array may then sit elsewhere.
struct NoAllocAddr {
    CUcontext ctx;
    cplx *ptr;
};
std::mutex g_noalloc_mu;
NoAllocAddr g_noalloc_addr[kNoAllocMaxDevices] = {};

yf_status current_context(CUcontext *ctx)
{
    static PFN_cuCtxGetCurrent_v4000 get = nullptr;
    if (!get) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(YF_E_CUDA, "yf_sparams_noalloc: cuCtxGetCurrent is not available");
        get = (PFN_cuCtxGetCurrent_v4000)fn;
    }
    if (get(ctx) != CUDA_SUCCESS || !*ctx)
        return fail(YF_E_CUDA, "yf_sparams_noalloc: no current CUDA context");
    return YF_OK;
}

// The array's device address in the current context.  A call outside stream capture looks
// it up (cheap once the module is loaded) and records it with the context; a call while
// `s` is capturing uses the recorded address, which must come from the same context.
yf_status noalloc_scratch(cudaStream_t s, cplx **out)
{
    int dev = -1;
    YF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(YF_E_UNSUPPORTED, "yf_sparams_noalloc: device %d beyond the %d supported", dev,
                    kNoAllocMaxDevices);
    CUcontext ctx = nullptr;
    yf_status st = current_context(&ctx);
    if (st != YF_OK) return st;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    YF_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocAddr &a = g_noalloc_addr[dev];
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_sstar);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_sstar)");
        a.ctx = ctx;
        a.ptr = (cplx *)p;
    } else if (!a.ptr || a.ctx != ctx) {
        return fail(YF_E_STATE, "yf_sparams_noalloc: the first call in a CUDA context (device %d) "
                                "must come before any stream capture", dev);
    }
    *out = a.ptr;
    return YF_OK;
}

}  // namespace
}  // namespace yf

extern "C" yf_status yf_sparams_noalloc(int nports, int nfreq, const double *freqs,
                                        const double *V_inc, const double *I_inc,
                                        const double *V_tot, double z_ref, double *S_star,
                                        double *S, double *Zr, double *Zc, double *tau,
                                        void *stream)
{
    using namespace yf;
    if (nports < 1 || nports > kMaxN || nfreq < 1 || !(z_ref > 0))
        return fail(YF_E_INVALID, "yf_sparams_noalloc: need 1 <= nports <= %d, nfreq >= 1, z_ref > 0",
                    kMaxN);
    if (!freqs || !V_inc || !I_inc || !V_tot || !S || !Zr)
        return fail(YF_E_INVALID, "yf_sparams_noalloc: freqs, V_inc, I_inc, V_tot, S and Zr are required");
    const long entries = (long)nfreq * nports * nports;
    if (entries > kNoAllocMaxEntries)
        return fail(YF_E_INVALID,
                    "yf_sparams_noalloc: nfreq * nports^2 = %ld exceeds the fixed scratch of %d entries",
                    entries, kNoAllocMaxEntries);
    cudaStream_t s = (cudaStream_t)stream;
    // an error left by earlier, unrelated work is reported before anything is queued, so a
    // failure here always means that this call wrote none of its outputs
    YF_CUDA_TRY(cudaGetLastError());
    cplx *scratch = nullptr;
    yf_status st = noalloc_scratch(s, &scratch);
    if (st != YF_OK) return st;
    SpArgs A;
    A.n = nports; A.nf = nfreq; A.uniform = 0; A.dir1 = 1; A.z_ref = z_ref;
    A.vinc = (const cplx *)V_inc;
    A.iinc = (const cplx *)I_inc;
    A.vtot = (const cplx *)V_tot;
    A.sstar = scratch;            // fully rewritten by every call: nothing to clear
    A.s = (cplx *)S;
    A.zr = (cplx *)Zr;
    A.zc = (nports == 2) ? (cplx *)Zc : nullptr;
    k_sparams<<<(nfreq + 63) / 64, 64, 0, s>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "yf_sparams_noalloc: k_sparams launch");
    if (tau) {
        k_phase_delay<<<1, 64, 0, s>>>(scratch, freqs, nports, nfreq, tau);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return cuda_fail(e, "yf_sparams_noalloc: k_phase_delay launch (S, Zr, Zc queued)");
    }
    if (S_star)
        YF_CUDA_TRY(cudaMemcpyAsync(S_star, scratch, (size_t)entries * sizeof(cplx),
                                    cudaMemcpyDeviceToDevice, s));
    return YF_OK;
}
