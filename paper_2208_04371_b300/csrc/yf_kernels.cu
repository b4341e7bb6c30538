// Reference-form Yee kernels (one thread per (i, j, k), in place), the per-step port
// epilogue (soft source, V / I integrals, running DFT) and the energy monitor.
//
// Yee leapfrog (Sec. II-A cites Yee 1966):
//   H^{n+1/2} = H^{n-1/2} - dt/mu0 curl E^n          (forward differences)
//   E^{n+1}   = Ca E^n + Cb curl H^{n+1/2}           (backward differences)
// with CPML auxiliaries inside the absorbing slabs (Sec. II-A cites Berenger's PML):
//   psi = b psi + a dF,   dF -> dF / kappa + psi.
#include <cuda_runtime.h>

#include "yf_internal.h"

namespace yf {
namespace {

__device__ __forceinline__ int slab_index(int p, int N, int n, int lo, int hi)
{
    if (lo && p < n) return p;
    if (hi && p >= N - n) return n + p - (N - n);
    return -1;
}

// CPML correction of one derivative: returns dF / kappa + psi_new and stores psi_new.
template <typename T>
__device__ __forceinline__ T cpml(T d, T *psi, const T *prof, int N1, int which, int p)
{
    // which = 0: integer-node profile (E updates), 3: half-node profile (H updates)
    const T b = prof[(which + 0) * N1 + p];
    const T a = prof[(which + 1) * N1 + p];
    const T rk = prof[(which + 2) * N1 + p];
    const T v = b * (*psi) + a * d;
    *psi = v;
    return d * rk + v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_update_h(StencilParams<T> P, Fields<T> F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i > P.nx || j > P.ny) return;
    const long q = (long)k * P.plane + (long)j * P.px + i;
    const T *ex = F.c[0], *ey = F.c[1], *ez = F.c[2];
    T *hx = F.c[3], *hy = F.c[4], *hz = F.c[5];
    const Pml<T> &M = P.pml;
    const int n = M.n, L = M.len;
    const int NX1 = P.nx + 1, NY1 = P.ny + 1, NZ1 = P.nz + 1;
    const int sx = slab_index(i, P.nx, n, M.lo[0], M.hi[0]);
    const int sy = slab_index(j, P.ny, n, M.lo[1], M.hi[1]);
    const int sz = slab_index(k, P.nz, n, M.lo[2], M.hi[2]);

    // H_x(i, j+1/2, k+1/2) -= dt/mu0 (dEz/dy - dEy/dz)
    if (j < P.ny && k < P.nz) {
        T d1 = (ez[q + P.px] - ez[q]) * P.rdy;
        T d2 = (ey[q + P.plane] - ey[q]) * P.rdz;
        if (sy >= 0) d1 = cpml(d1, M.psi[1][2] + ((long)k * L + sy) * P.px + i, M.prof[1], NY1, 3, j);
        if (sz >= 0) d2 = cpml(d2, M.psi[2][2] + ((long)sz * NY1 + j) * P.px + i, M.prof[2], NZ1, 3, k);
        hx[q] -= P.db * (d1 - d2);
    }
    // H_y(i+1/2, j, k+1/2) -= dt/mu0 (dEx/dz - dEz/dx)
    if (i < P.nx && k < P.nz) {
        T d1 = (ex[q + P.plane] - ex[q]) * P.rdz;
        T d2 = (ez[q + 1] - ez[q]) * P.rdx;
        if (sz >= 0) d1 = cpml(d1, M.psi[2][3] + ((long)sz * NY1 + j) * P.px + i, M.prof[2], NZ1, 3, k);
        if (sx >= 0) d2 = cpml(d2, M.psi[0][2] + ((long)k * NY1 + j) * L + sx, M.prof[0], NX1, 3, i);
        hy[q] -= P.db * (d1 - d2);
    }
    // H_z(i+1/2, j+1/2, k) -= dt/mu0 (dEy/dx - dEx/dy)
    if (i < P.nx && j < P.ny) {
        T d1 = (ey[q + 1] - ey[q]) * P.rdx;
        T d2 = (ex[q + P.px] - ex[q]) * P.rdy;
        if (sx >= 0) d1 = cpml(d1, M.psi[0][3] + ((long)k * NY1 + j) * L + sx, M.prof[0], NX1, 3, i);
        if (sy >= 0) d2 = cpml(d2, M.psi[1][3] + ((long)k * L + sy) * P.px + i, M.prof[1], NY1, 3, j);
        hz[q] -= P.db * (d1 - d2);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_update_e(StencilParams<T> P, Fields<T> F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i > P.nx || j > P.ny) return;
    const long q = (long)k * P.plane + (long)j * P.px + i;
    T *ex = F.c[0], *ey = F.c[1], *ez = F.c[2];
    const T *hx = F.c[3], *hy = F.c[4], *hz = F.c[5];
    const Pml<T> &M = P.pml;
    const int n = M.n, L = M.len;
    const int NX1 = P.nx + 1, NY1 = P.ny + 1, NZ1 = P.nz + 1;
    const int sx = slab_index(i, P.nx, n, M.lo[0], M.hi[0]);
    const int sy = slab_index(j, P.ny, n, M.lo[1], M.hi[1]);
    const int sz = slab_index(k, P.nz, n, M.lo[2], M.hi[2]);

    // E_x(i+1/2, j, k) = Ca E_x + Cb (dHz/dy - dHy/dz); tangential on the walls stays 0
    if (i < P.nx && j >= 1 && j < P.ny && k >= 1 && k < P.nz) {
        const int c = P.cls[0][q];
        if (c) {
            T d1 = (hz[q] - hz[q - P.px]) * P.rdy;
            T d2 = (hy[q] - hy[q - P.plane]) * P.rdz;
            if (sy >= 0) d1 = cpml(d1, M.psi[1][0] + ((long)k * L + sy) * P.px + i, M.prof[1], NY1, 0, j);
            if (sz >= 0) d2 = cpml(d2, M.psi[2][0] + ((long)sz * NY1 + j) * P.px + i, M.prof[2], NZ1, 0, k);
            ex[q] = P.ctab[2 * c] * ex[q] + P.ctab[2 * c + 1] * (d1 - d2);
        }
    }
    // E_y(i, j+1/2, k) = Ca E_y + Cb (dHx/dz - dHz/dx)
    if (i >= 1 && i < P.nx && j < P.ny && k >= 1 && k < P.nz) {
        const int c = P.cls[1][q];
        if (c) {
            T d1 = (hx[q] - hx[q - P.plane]) * P.rdz;
            T d2 = (hz[q] - hz[q - 1]) * P.rdx;
            if (sz >= 0) d1 = cpml(d1, M.psi[2][1] + ((long)sz * NY1 + j) * P.px + i, M.prof[2], NZ1, 0, k);
            if (sx >= 0) d2 = cpml(d2, M.psi[0][0] + ((long)k * NY1 + j) * L + sx, M.prof[0], NX1, 0, i);
            ey[q] = P.ctab[2 * c] * ey[q] + P.ctab[2 * c + 1] * (d1 - d2);
        }
    }
    // E_z(i, j, k+1/2) = Ca E_z + Cb (dHy/dx - dHx/dy)
    if (i >= 1 && i < P.nx && j >= 1 && j < P.ny && k < P.nz) {
        const int c = P.cls[2][q];
        if (c) {
            T d1 = (hy[q] - hy[q - 1]) * P.rdx;
            T d2 = (hx[q] - hx[q - P.px]) * P.rdy;
            if (sx >= 0) d1 = cpml(d1, M.psi[0][1] + ((long)k * NY1 + j) * L + sx, M.prof[0], NX1, 0, i);
            if (sy >= 0) d2 = cpml(d2, M.psi[1][1] + ((long)k * L + sy) * P.px + i, M.prof[1], NY1, 0, j);
            ez[q] = P.ctab[2 * c] * ez[q] + P.ctab[2 * c + 1] * (d1 - d2);
        }
    }
}

// ---------------------------------------------------------------------------------------
// per-step epilogue: one block

__device__ double waveform(int kind, double p0, double p1, double t0, const double *table,
                           long table_len, long long n_plus_1, double dt)
{
    const double t = (double)n_plus_1 * dt;
    if (kind == YF_WAVE_DIFF_GAUSS) {        // Eq. 3
        const double u = (t - t0) / p0;
        return -2.0 * u * exp(-u * u);
    }
    if (kind == YF_WAVE_GAUSS_SINE) {
        const double tau = 2.0 / (3.14159265358979323846 * p1);
        const double u = t - t0;
        return sin(2.0 * 3.14159265358979323846 * p0 * u) * exp(-(u / tau) * (u / tau));
    }
    if (kind == YF_WAVE_TABLE) return (n_plus_1 - 1 < table_len) ? table[n_plus_1 - 1] : 0.0;
    return 0.0;
}

// Deterministic block sum (fixed shuffle tree, then warp partials in order).
__device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;   // valid in thread 0
}

__device__ __forceinline__ void kahan_add(float *sum, float *comp, float x)
{
    const float y = x - *comp;
    const float t = *sum + y;
    *comp = (t - *sum) - y;
    *sum = t;
}

// One work item of the epilogue: kind 0 adds the source on its points; kinds 1 and 2 return
// the block's partial V or I sum (valid in thread 0).
template <typename T>
__device__ double epi_segment(const EpiParams<T> &P, const EpiSeg &S, long long n, double *red)
{
    const int tid = threadIdx.x;
    if (S.kind == 0) {
        // soft source E_z += A s(t_{n+1}) on plane e (Eq. 3)
        const double s = waveform(P.src_kind, P.p0, P.p1, P.t0, P.table, P.table_len, n + 1, P.dt);
        const T add = (T)(P.amp * s);
        const int nj = P.sj1 - P.sj0 + 1;
        for (int w = S.start + tid; w < S.start + S.count; w += blockDim.x) {
            const int j = P.sj0 + w % nj, k = P.sk0 + w / nj;
            const long q = (long)k * P.plane + (long)j * P.px + P.src_plane;
            if (P.cls_z[q]) P.ez[q] += add;
        }
        return 0.0;
    }
    const PortDev d = P.ports[S.port];
    double acc = 0.0;
    if (S.kind == 1) {
        // V: surface integral of E_z across the strip (Eq. 4), trapezoid in y
        const int nj = d.j1 - d.j0 + 1;
        for (int w = S.start + tid; w < S.start + S.count; w += blockDim.x) {
            const int j = d.j0 + w % nj, k = d.k0 + w / nj;
            const double wj = (j == d.j0 || j == d.j1) ? 0.5 : 1.0;
            acc += wj * (double)P.ez[(long)k * P.plane + (long)j * P.px + d.plane];
        }
    } else {
        // I: loops of H at x = plane - 1/2 and plane + 1/2 (Eq. 4)
        const int nyl = d.j1 - d.j0 + 2 * d.m - 1, nzl = d.kt - d.kb + 2 * d.m - 1;
        const int per = 2 * nyl + 2 * nzl;
        for (int w = S.start + tid; w < S.start + S.count; w += blockDim.x) {
            const int ih = d.plane - 1 + w / per;
            const int r = w % per;
            if (r < 2 * nyl) {
                const int j = d.j0 - d.m + 1 + (r >> 1);
                if ((r & 1) == 0)   // bottom, along +y
                    acc += (double)P.hy[(long)(d.kb - d.m) * P.plane + (long)j * P.px + ih] * P.dy;
                else                // top, along -y
                    acc -= (double)P.hy[(long)(d.kt + d.m - 1) * P.plane + (long)j * P.px + ih] * P.dy;
            } else {
                const int r2 = r - 2 * nyl;
                const int k = d.kb - d.m + 1 + (r2 >> 1);
                if ((r2 & 1) == 0)  // right side, along +z
                    acc += (double)P.hz[(long)k * P.plane + (long)(d.j1 + d.m - 1) * P.px + ih] * P.dz;
                else                // left side, along -z
                    acc -= (double)P.hz[(long)k * P.plane + (long)(d.j0 - d.m) * P.px + ih] * P.dz;
            }
        }
    }
    return block_sum(acc, red);
}

// Running DFT with exact integer phase (V at 2(n+1) half steps, I at 2n+1), then the
// finite check and the step counter; vi holds each port's V and I.
template <typename T>
__device__ void epi_finish(const EpiParams<T> &P, long long n, const double (*vi)[2])
{
    const int tid = threadIdx.x;
    int total = 0;
    for (int p = 0; p < P.nports; ++p) total += P.ports[p].nfreq;
    for (int w = tid; w < total; w += blockDim.x) {
        int p = 0;
        while (p + 1 < P.nports && w >= P.ports[p + 1].foff) ++p;
        const double V = vi[p][0], I = vi[p][1];
        const unsigned long long inc = P.inc[w];
        const unsigned long long phv = (unsigned long long)(2 * (n + 1)) * inc;
        const unsigned long long phi = (unsigned long long)(2 * n + 1) * inc;
        double sv, cv, si, ci;
        sincospi((double)(long long)phv * 0x1p-63, &sv, &cv);
        sincospi((double)(long long)phi * 0x1p-63, &si, &ci);
        const double t0 = V * cv, t1 = -V * sv, t2 = I * ci, t3 = -I * si;
        if (P.dft_mask & YF_DFT_FP64) {
            double *a = P.acc64 + 4 * (long)w;
            a[0] += t0; a[1] += t1; a[2] += t2; a[3] += t3;
        }
        if (P.dft_mask & YF_DFT_FP32) {
            float *a = P.acc32 + 4 * (long)w;
            a[0] += (float)t0; a[1] += (float)t1; a[2] += (float)t2; a[3] += (float)t3;
        }
        if (P.dft_mask & YF_DFT_KAHAN32) {
            float *a = P.kahan + 8 * (long)w;
            kahan_add(a + 0, a + 1, (float)t0);
            kahan_add(a + 2, a + 3, (float)t1);
            kahan_add(a + 4, a + 5, (float)t2);
            kahan_add(a + 6, a + 7, (float)t3);
        }
    }
    __syncthreads();
    if (tid == 0) {
        int bad = 0;
        for (int p = 0; p < P.nports; ++p)
            if (!isfinite(vi[p][0]) || !isfinite(vi[p][1])) bad = 1;
        if (bad) atomicOr(P.status, 1);
        *P.ctr = n + 1;
        if (!P.skip_source) *P.src_ctr = n + 1;
    }
}

template <typename T>
__device__ void epi_scale(const EpiParams<T> &P, double (*vi)[2])
{
    for (int p = 0; p < P.nports; ++p) {
        const PortDev d = P.ports[p];
        vi[p][0] = d.vscale * vi[p][0];
        vi[p][1] = (double)d.dir * 0.5 * vi[p][1];
    }
}

// Single grid: the segments are spread over the blocks; each V/I partial lands in its own
// slot and the last block to arrive combines them in segment order (deterministic).
template <typename T>
__global__ void __launch_bounds__(kEpiThreads) k_epilogue(EpiParams<T> P)
{
    __shared__ double red[kEpiThreads / 32];
    __shared__ double vi[kMaxPorts][2];
    __shared__ double pval[kEpiThreads];
    __shared__ int pdst[kEpiThreads];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const long long n = *P.ctr;   // this is step n: E^{n+1}, H^{n+1/2} are in place
    for (int sg = blockIdx.x; sg < P.nseg; sg += gridDim.x) {
        if (P.skip_source && P.segs[sg].kind == 0) continue;
        const double part = epi_segment(P, P.segs[sg], n, red);
        if (tid == 0 && P.segs[sg].kind != 0) P.slots[sg] = part;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(P.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (tid == 0)
        for (int p = 0; p < P.nports; ++p) { vi[p][0] = 0.0; vi[p][1] = 0.0; }
    // the block fetches the partials of up to kEpiThreads segments at once; thread 0 adds them
    // in segment order
    for (int c = 0; c < P.nseg; c += kEpiThreads) {
        const int sg = c + tid;
        int dst = -1;
        double v = 0.0;
        if (sg < P.nseg) {
            const EpiSeg S = P.segs[sg];
            if (S.kind != 0) {
                dst = 2 * S.port + (S.kind == 2);
                v = __ldcg(P.slots + sg);
            }
        }
        pdst[tid] = dst;
        pval[tid] = v;
        __syncthreads();
        if (tid == 0) {
            const int m = P.nseg - c < kEpiThreads ? P.nseg - c : kEpiThreads;
            for (int q = 0; q < m; ++q)
                if (pdst[q] >= 0) vi[pdst[q] >> 1][pdst[q] & 1] += pval[q];
        }
        __syncthreads();
    }
    if (tid == 0) {
        epi_scale(P, vi);
        *P.ticket = 0;
    }
    __syncthreads();
    epi_finish(P, n, vi);
}

// The soft source alone (Eq. 3), for the path that runs the port integrals and transforms on
// a side stream: it is the only part of the epilogue that the next step reads.  One thread per
// point of the source rectangle; each block evaluates the waveform once; its own step counter,
// advanced by the last block to finish (ticket[1]), so that it may run ahead of the transforms.
template <typename T>
__global__ void __launch_bounds__(kEpiThreads) k_epi_source(EpiParams<T> P)
{
    __shared__ T add;
    __shared__ bool last;
    const long long n = *P.src_ctr;
    if (threadIdx.x == 0)
        add = (T)(P.amp * waveform(P.src_kind, P.p0, P.p1, P.t0, P.table, P.table_len, n + 1, P.dt));
    __syncthreads();
    const int nj = P.sj1 - P.sj0 + 1, npt = P.src_kind == YF_WAVE_NONE ? 0 : nj * (P.sk1 - P.sk0);
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < npt; w += gridDim.x * blockDim.x) {
        const int j = P.sj0 + w % nj, k = P.sk0 + w / nj;
        const long q = (long)k * P.plane + (long)j * P.px + P.src_plane;
        if (P.cls_z[q]) P.ez[q] += add;
    }
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(P.ticket + 1, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last && threadIdx.x == 0) {
        P.ticket[1] = 0;
        *P.src_ctr = n + 1;
    }
}

// Many grids: block b runs the whole epilogue of grid b (parameters of the current parity).
template <typename T>
__global__ void __launch_bounds__(kEpiThreads) k_epilogue_batch(const EpiParams<T> *eps, int parity, int stride)
{
    __shared__ double red[kEpiThreads / 32];
    __shared__ double vi[kMaxPorts][2];
    const EpiParams<T> P = eps[stride * blockIdx.x + parity];
    const int tid = threadIdx.x;
    const long long n = *P.ctr;
    if (tid == 0)
        for (int p = 0; p < P.nports; ++p) { vi[p][0] = 0.0; vi[p][1] = 0.0; }
    for (int sg = 0; sg < P.nseg; ++sg) {
        const EpiSeg S = P.segs[sg];
        const double part = epi_segment(P, S, n, red);
        if (tid == 0) {
            if (S.kind == 1) vi[S.port][0] += part;
            else if (S.kind == 2) vi[S.port][1] += part;
        }
    }
    if (tid == 0) epi_scale(P, vi);
    __syncthreads();
    epi_finish(P, n, vi);
}

// ---------------------------------------------------------------------------------------
// energy monitor: partial sums per block (fixed grid), then one ordered final sum

template <typename T>
struct EnergyArgs {
    const T *c[6];
    const uint8_t *cls[3];
    const double *eps_tab;
    long npts;
};

template <typename T>
__global__ void __launch_bounds__(256) k_energy_partial(EnergyArgs<T> A, double *partials)
{
    __shared__ double red[8];
    double w = 0.0;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < A.npts;
         q += (long)gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; ++c) {
            const int cl = A.cls[c][q];
            if (cl) {
                const double e = (double)A.c[c][q];
                w += A.eps_tab[cl] * e * e;
            }
        }
        for (int c = 3; c < 6; ++c) {
            const double h = (double)A.c[c][q];
            w += kMu0 * h * h;
        }
    }
    const double s = block_sum(w, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_energy_final(const double *partials, int n, double *out)
{
    __shared__ double red[8];
    double w = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) w += partials[b];
    const double s = block_sum(w, red);
    if (threadIdx.x == 0) *out = s;
}

// Zero what the update never writes: E on class-0 (PEC, wall) edges and H outside
// each component's index range.
template <typename T>
__global__ void k_sanitize(Fields<T> F, const uint8_t *cx, const uint8_t *cy, const uint8_t *cz,
                           int nx, int ny, int nz, int px, long plane)
{
    const long npts = plane * (nz + 1);
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < npts;
         q += (long)gridDim.x * blockDim.x) {
        const int k = (int)(q / plane);
        const int r = (int)(q % plane);
        const int j = r / px, i = r % px;
        if (!cx[q]) F.c[0][q] = (T)0;
        if (!cy[q]) F.c[1][q] = (T)0;
        if (!cz[q]) F.c[2][q] = (T)0;
        if (!(i <= nx && j < ny && k < nz)) F.c[3][q] = (T)0;
        if (!(i < nx && j <= ny && k < nz)) F.c[4][q] = (T)0;
        if (!(i < nx && j < ny && k <= nz)) F.c[5][q] = (T)0;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_epi_source(const EpiParams<T> &p, cudaStream_t s)
{
    const int npt = p.src_kind == YF_WAVE_NONE ? 0 : (p.sj1 - p.sj0 + 1) * (p.sk1 - p.sk0);
    const int nblk = npt < kEpiThreads ? 1 : (npt + kEpiThreads - 1) / kEpiThreads;
    k_epi_source<T><<<nblk < 296 ? nblk : 296, kEpiThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_epilogue_batch(const EpiParams<T> *eps, int n, int parity, cudaStream_t s, int stride)
{
    if (n <= 0) return cudaSuccess;
    k_epilogue_batch<T><<<n, kEpiThreads, 0, s>>>(eps, parity, stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sanitize(const Fields<T> &f, uint8_t *const cls[3], int nx, int ny, int nz,
                            int px, long plane, cudaStream_t s)
{
    k_sanitize<T><<<1184, 256, 0, s>>>(f, cls[0], cls[1], cls[2], nx, ny, nz, px, plane);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_h(const StencilParams<T> &p, const Fields<T> &f, cudaStream_t s)
{
    dim3 blk(32, 8), grd((p.nx + 1 + 31) / 32, (p.ny + 1 + 7) / 8, p.nz + 1);
    k_update_h<T><<<grd, blk, 0, s>>>(p, f);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_e(const StencilParams<T> &p, const Fields<T> &f, cudaStream_t s)
{
    dim3 blk(32, 8), grd((p.nx + 1 + 31) / 32, (p.ny + 1 + 7) / 8, p.nz + 1);
    k_update_e<T><<<grd, blk, 0, s>>>(p, f);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_epilogue(const EpiParams<T> &p, cudaStream_t s)
{
    const int nblk = p.nseg < 1 ? 1 : (p.nseg < 296 ? p.nseg : 296);
    k_epilogue<T><<<nblk, kEpiThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_energy(const T *const c[6], const uint8_t *const cls[3], const double *eps_tab,
                          int nx, int ny, int nz, int px, long plane, double *partials,
                          double *out, cudaStream_t s)
{
    EnergyArgs<T> A;
    for (int q = 0; q < 6; ++q) A.c[q] = c[q];
    for (int q = 0; q < 3; ++q) A.cls[q] = cls[q];
    A.eps_tab = eps_tab;
    A.npts = plane * (long)(nz + 1);
    (void)nx; (void)ny; (void)px;
    k_energy_partial<T><<<kEnergyBlocks, 256, 0, s>>>(A, partials);
    k_energy_final<<<1, 256, 0, s>>>(partials, kEnergyBlocks, out);
    return cudaGetLastError();
}

#define YF_INST(T)                                                                          \
    template cudaError_t launch_update_h<T>(const StencilParams<T> &, const Fields<T> &,     \
                                            cudaStream_t);                                  \
    template cudaError_t launch_update_e<T>(const StencilParams<T> &, const Fields<T> &,     \
                                            cudaStream_t);                                  \
    template cudaError_t launch_epilogue<T>(const EpiParams<T> &, cudaStream_t);            \
    template cudaError_t launch_epi_source<T>(const EpiParams<T> &, cudaStream_t);          \
    template cudaError_t launch_epilogue_batch<T>(const EpiParams<T> *, int, int, cudaStream_t, int); \
    template cudaError_t launch_sanitize<T>(const Fields<T> &, uint8_t *const[3], int, int, \
                                            int, int, long, cudaStream_t);                  \
    template cudaError_t launch_energy<T>(const T *const[6], const uint8_t *const[3],        \
                                          const double *, int, int, int, int, long,          \
                                          double *, double *, cudaStream_t);
YF_INST(float)
YF_INST(double)

}  // namespace yf
