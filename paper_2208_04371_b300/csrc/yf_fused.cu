// Fused Yee step: H^{n+1/2} and E^{n+1} in one pass over HBM.
//
// Each block owns a TX x TY column of (i, j) nodes and marches a segment of z-planes.  The
// step reads buffer A (E^n, H^{n-1/2}) and writes buffer B (E^{n+1}, H^{n+1/2}), so blocks
// never see each other's writes and no grid-wide ordering is needed.  Per plane p the block
//   1. stages the (TX+2) x (TY+2) window of E^n on plane p+1 in shared memory (plane p is
//      already there from the previous iteration);
//   2. computes H^{n+1/2} on plane p for its nodes plus the low halo row j0-1 and column
//      i0-1 (recomputed, not stored) that the E update needs, writes its own H to B;
//   3. computes E^{n+1} on plane p from those H values and H^{n+1/2} of plane p-1 (kept in
//      registers from the previous iteration), writes it to B.
// A segment starting at plane kb > 0 first recomputes H_x, H_y of plane kb-1 (not stored).
// CPML: the E auxiliaries are updated in place (only the owner touches them); the H
// auxiliaries are read from one copy and written to the other, because halo H values of a
// neighbour's nodes are recomputed from the old auxiliaries.
#include <cuda_runtime.h>

#include "yf_internal.h"

namespace yf {
namespace {

__device__ __forceinline__ int slab_idx(int p, int N, int n, int lo, int hi)
{
    if (lo && p < n) return p;
    if (hi && p >= N - n) return n + p - (N - n);
    return -1;
}

// psi_new = b psi_old + a d; returns d / kappa + psi_new.  w may be null (halo nodes).
template <typename T>
__device__ __forceinline__ T cpml_rw(T d, const T *r, T *w, const T *prof, int N1, int which, int p)
{
    const T b = prof[(which + 0) * N1 + p];
    const T a = prof[(which + 1) * N1 + p];
    const T rk = prof[(which + 2) * N1 + p];
    const T v = b * (*r) + a * d;
    if (w) *w = v;
    return d * rk + v;
}

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, 1024 / (TX * TY)) k_yee_fused(FusedArgs<T> P)
{
    constexpr int WX = TX + 2, WY = TY + 2, WN = WX * WY;
    constexpr int NT = TX * TY;
    constexpr int R = (3 * WN + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sE = reinterpret_cast<T *>(smraw);   // [2][3][WN]: E^n on planes p (cur) and p+1
    T *sH = sE + 6 * WN;                     // [3][WN]: H^{n+1/2} on plane p
    T *sC = sH + 3 * WN;                     // [2 * kMaxClasses]: (Ca, Cb)

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = (blockIdx.x + P.tx0) * TX, j0 = (blockIdx.y + P.ty0) * TY;
    const int i = i0 + tx, j = j0 + ty;
    const int kb = P.z0 + blockIdx.z * P.kseg;
    if (kb > P.z1) return;
    const int ke = min(P.z1, kb + P.kseg - 1);
    const long plane = P.plane, npts = P.npts;
    const int px = P.px, NX1 = P.nx + 1, NY1 = P.ny + 1, NZ1 = P.nz + 1;
    const int n = P.n, L = P.L;

    for (int q = tid; q < 2 * kMaxClasses; q += NT) sC[q] = P.ctab[q];

    // stage the E window (3 components, (TX+2) x (TY+2) nodes) of plane kp in buffer buf;
    // nodes outside the grid read as zero
    auto load_plane = [&](int buf, int kp) {
        const bool kin = kp >= 0 && kp <= P.nz;
        const T *src = P.A + (long)(kin ? kp : 0) * plane;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int q = tid + r * NT;
            if (q < 3 * WN) {
                const int c = q / WN, rr = q - c * WN;
                const int jj = rr / WX, ii = rr - jj * WX;
                const int gi = i0 - 1 + ii, gj = j0 - 1 + jj;
                T v = 0;
                if (kin && gi >= 0 && gi < px && gj >= 0 && gj <= P.ny)
                    v = ldg(src + (long)c * npts + (long)gj * px + gi);
                sE[buf * 3 * WN + q] = v;
            }
        }
    };

    // slab indices that do not change along the march
    const int sx_own = slab_idx(i, P.nx, n, P.lo[0], P.hi[0]);
    const int sy_own = slab_idx(j, P.ny, n, P.lo[1], P.hi[1]);
    const bool live = i <= P.nx && j <= P.ny;
    const int wown = (ty + 1) * WX + (tx + 1);

    T hx_prev = 0, hy_prev = 0;
    int cur = 0;
    load_plane(cur, kb - 1);

    for (int p = kb - 1; p <= ke; ++p) {
        const int nxt = cur ^ 1;
        load_plane(nxt, p + 1);
        const bool pin = p >= 0;
        const long pbase = (long)(pin ? p : 0) * plane;
        // H^{n-1/2} on plane p at the own node and at the halo nodes this thread computes
        T hxo = 0, hyo = 0, hzo = 0;
        if (pin && live) {
            const long q = pbase + (long)j * px + i;
            hxo = ldg(P.A + 3 * npts + q);
            hyo = ldg(P.A + 4 * npts + q);
            hzo = ldg(P.A + 5 * npts + q);
        }
        T hrow_x = 0, hrow_z = 0, hcol_y = 0, hcol_z = 0;
        const bool do_row = ty == 0 && j0 > 0 && i <= P.nx && p >= kb;
        const bool do_col = tx == 0 && i0 > 0 && j <= P.ny && p >= kb;
        if (do_row) {
            const long q = pbase + (long)(j0 - 1) * px + i;
            hrow_x = ldg(P.A + 3 * npts + q);
            hrow_z = ldg(P.A + 5 * npts + q);
        }
        if (do_col) {
            const long q = pbase + (long)j * px + (i0 - 1);
            hcol_y = ldg(P.A + 4 * npts + q);
            hcol_z = ldg(P.A + 5 * npts + q);
        }
        __syncthreads();

        const T *ex0 = sE + cur * 3 * WN, *ey0 = ex0 + WN, *ez0 = ey0 + WN;
        const T *ex1 = sE + nxt * 3 * WN, *ey1 = ex1 + WN;
        const int sz = pin ? slab_idx(p, P.nz, n, P.lo[2], P.hi[2]) : -1;

        // H at window node w (global i_, j_) on plane p; own = write the H auxiliaries
        auto hx_at = [&](int w, int i_, int j_, int sy_, bool own, T old) -> T {
            T d1 = (ez0[w + WX] - ez0[w]) * P.rdy;
            T d2 = (ey1[w] - ey0[w]) * P.rdz;
            if (sy_ >= 0) {
                const long o = ((long)p * L + sy_) * px + i_;
                d1 = cpml_rw(d1, P.psiHr[1][0] + o, own ? P.psiHw[1][0] + o : (T *)nullptr, P.prof[1], NY1, 3, j_);
            }
            if (sz >= 0) {
                const long o = ((long)sz * NY1 + j_) * px + i_;
                d2 = cpml_rw(d2, P.psiHr[2][0] + o, own ? P.psiHw[2][0] + o : (T *)nullptr, P.prof[2], NZ1, 3, p);
            }
            return old - P.db * (d1 - d2);
        };
        auto hy_at = [&](int w, int i_, int j_, int sx_, bool own, T old) -> T {
            T d1 = (ex1[w] - ex0[w]) * P.rdz;
            T d2 = (ez0[w + 1] - ez0[w]) * P.rdx;
            if (sz >= 0) {
                const long o = ((long)sz * NY1 + j_) * px + i_;
                d1 = cpml_rw(d1, P.psiHr[2][1] + o, own ? P.psiHw[2][1] + o : (T *)nullptr, P.prof[2], NZ1, 3, p);
            }
            if (sx_ >= 0) {
                const long o = ((long)p * NY1 + j_) * L + sx_;
                d2 = cpml_rw(d2, P.psiHr[0][0] + o, own ? P.psiHw[0][0] + o : (T *)nullptr, P.prof[0], NX1, 3, i_);
            }
            return old - P.db * (d1 - d2);
        };
        auto hz_at = [&](int w, int i_, int j_, int sx_, int sy_, bool own, T old) -> T {
            T d1 = (ey0[w + 1] - ey0[w]) * P.rdx;
            T d2 = (ex0[w + WX] - ex0[w]) * P.rdy;
            if (sx_ >= 0) {
                const long o = ((long)p * NY1 + j_) * L + sx_;
                d1 = cpml_rw(d1, P.psiHr[0][1] + o, own ? P.psiHw[0][1] + o : (T *)nullptr, P.prof[0], NX1, 3, i_);
            }
            if (sy_ >= 0) {
                const long o = ((long)p * L + sy_) * px + i_;
                d2 = cpml_rw(d2, P.psiHr[1][1] + o, own ? P.psiHw[1][1] + o : (T *)nullptr, P.prof[1], NY1, 3, j_);
            }
            return old - P.db * (d1 - d2);
        };

        if (p < kb) {
            // warm-up plane kb - 1: own H_x, H_y only (the E update of plane kb needs them)
            if (pin && live && p < P.nz) {
                hx_prev = hx_at(wown, i, j, sy_own, false, hxo);
                hy_prev = hy_at(wown, i, j, sx_own, false, hyo);
            }
        } else {
            // own node
            const bool vx = live && j < P.ny && p < P.nz;
            const bool vy = live && i < P.nx && p < P.nz;
            const bool vz = live && i < P.nx && j < P.ny;
            T hx = 0, hy = 0, hz = 0;
            if (live) {
                hx = hx_at(wown, i, j, sy_own, vx, hxo);
                hy = hy_at(wown, i, j, sx_own, vy, hyo);
                hz = hz_at(wown, i, j, sx_own, sy_own, vz, hzo);
            }
            sH[0 * WN + wown] = hx;
            sH[1 * WN + wown] = hy;
            sH[2 * WN + wown] = hz;
            // halo row j0-1 (H_x, H_z) and column i0-1 (H_y, H_z)
            if (ty == 0) {
                const int w = tx + 1;   // jj = 0
                T a = 0, b = 0;
                if (do_row) {
                    const int sy_ = slab_idx(j0 - 1, P.ny, n, P.lo[1], P.hi[1]);
                    a = hx_at(w, i, j0 - 1, sy_, false, hrow_x);
                    b = hz_at(w, i, j0 - 1, sx_own, sy_, false, hrow_z);
                }
                sH[0 * WN + w] = a;
                sH[2 * WN + w] = b;
            }
            if (tx == 0) {
                const int w = (ty + 1) * WX;   // ii = 0
                T a = 0, b = 0;
                if (do_col) {
                    const int sx_ = slab_idx(i0 - 1, P.nx, n, P.lo[0], P.hi[0]);
                    a = hy_at(w, i0 - 1, j, sx_, false, hcol_y);
                    b = hz_at(w, i0 - 1, j, sx_, sy_own, false, hcol_z);
                }
                sH[1 * WN + w] = a;
                sH[2 * WN + w] = b;
            }
            if (live) {
                const long q = (long)p * plane + (long)j * px + i;
                if (vx) P.B[3 * npts + q] = hx;
                if (vy) P.B[4 * npts + q] = hy;
                if (vz) P.B[5 * npts + q] = hz;
            }
            __syncthreads();

            if (live) {
                const long q = (long)p * plane + (long)j * px + i;
                const T *shx = sH, *shy = sH + WN, *shz = sH + 2 * WN;
                T exn = 0, eyn = 0, ezn = 0;
                // E_x(i+1/2, j, p) = Ca E_x + Cb (dHz/dy - dHy/dz)
                int c = P.cls[0][q];
                if (c) {
                    T d1 = (shz[wown] - shz[wown - WX]) * P.rdy;
                    T d2 = (shy[wown] - hy_prev) * P.rdz;
                    if (sy_own >= 0) {
                        T *o = P.psiE[1][0] + ((long)p * L + sy_own) * px + i;
                        d1 = cpml_rw(d1, o, o, P.prof[1], NY1, 0, j);
                    }
                    if (sz >= 0) {
                        T *o = P.psiE[2][0] + ((long)sz * NY1 + j) * px + i;
                        d2 = cpml_rw(d2, o, o, P.prof[2], NZ1, 0, p);
                    }
                    exn = sC[2 * c] * ex0[wown] + sC[2 * c + 1] * (d1 - d2);
                }
                // E_y(i, j+1/2, p) = Ca E_y + Cb (dHx/dz - dHz/dx)
                c = P.cls[1][q];
                if (c) {
                    T d1 = (shx[wown] - hx_prev) * P.rdz;
                    T d2 = (shz[wown] - shz[wown - 1]) * P.rdx;
                    if (sz >= 0) {
                        T *o = P.psiE[2][1] + ((long)sz * NY1 + j) * px + i;
                        d1 = cpml_rw(d1, o, o, P.prof[2], NZ1, 0, p);
                    }
                    if (sx_own >= 0) {
                        T *o = P.psiE[0][0] + ((long)p * NY1 + j) * L + sx_own;
                        d2 = cpml_rw(d2, o, o, P.prof[0], NX1, 0, i);
                    }
                    eyn = sC[2 * c] * ey0[wown] + sC[2 * c + 1] * (d1 - d2);
                }
                // E_z(i, j, p+1/2) = Ca E_z + Cb (dHy/dx - dHx/dy)
                c = P.cls[2][q];
                if (c) {
                    T d1 = (shy[wown] - shy[wown - 1]) * P.rdx;
                    T d2 = (shx[wown] - shx[wown - WX]) * P.rdy;
                    if (sx_own >= 0) {
                        T *o = P.psiE[0][1] + ((long)p * NY1 + j) * L + sx_own;
                        d1 = cpml_rw(d1, o, o, P.prof[0], NX1, 0, i);
                    }
                    if (sy_own >= 0) {
                        T *o = P.psiE[1][1] + ((long)p * L + sy_own) * px + i;
                        d2 = cpml_rw(d2, o, o, P.prof[1], NY1, 0, j);
                    }
                    ezn = sC[2 * c] * ez0[wown] + sC[2 * c + 1] * (d1 - d2);
                }
                P.B[q] = exn;
                P.B[npts + q] = eyn;
                P.B[2 * npts + q] = ezn;
            }
            hx_prev = hx;
            hy_prev = hy;
        }
        __syncthreads();
        cur = nxt;
    }
}

template <typename T, int TX, int TY>
cudaError_t launch_fused_t(const FusedArgs<T> &a, cudaStream_t s)
{
    constexpr int WN = (TX + 2) * (TY + 2);
    const size_t smem = (9 * WN + 2 * kMaxClasses) * sizeof(T);
    dim3 blk(TX, TY), grd((a.nx + 1 + TX - 1) / TX, (a.ny + 1 + TY - 1) / TY,
                          (a.nz + 1 + a.kseg - 1) / a.kseg);
    k_yee_fused<T, TX, TY><<<grd, blk, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_fused(const FusedArgs<T> &a, int tile_y, cudaStream_t s)
{
    switch (tile_y) {
    case 4: return launch_fused_t<T, 32, 4>(a, s);
    case 16: return launch_fused_t<T, 32, 16>(a, s);
    default: return launch_fused_t<T, 32, 8>(a, s);
    }
}

template cudaError_t launch_fused<float>(const FusedArgs<float> &, int, cudaStream_t);
template cudaError_t launch_fused<double>(const FusedArgs<double> &, int, cudaStream_t);

}  // namespace yf
