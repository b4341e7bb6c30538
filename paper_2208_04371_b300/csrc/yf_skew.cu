// Fused Yee step, TMA-staged and skewed by one plane (variant 3).
//
// Same update as the other fused variants (buffer A -> buffer B, halo H recomputed).  The
// march is skewed: iteration t computes H^{n+1/2} on plane t (own nodes and the low halo row
// and column, into shared buffer t mod 2) and E^{n+1} on plane t - 1 (whose neighbour H
// values were finished in the previous iteration).  Both halves read only data completed
// before the iteration began, so one block barrier per plane suffices.  Plane q's E^n window,
// H^{n-1/2} window and edge classes arrive by TMA in stage (q - kb + 1) mod 4; a stage is
// used by iterations q - 1, q and q + 1 and refilled with plane q + 4 after iteration q + 1.
// The CPML auxiliaries a thread needs are loaded at the top of its iteration, so their
// latency overlaps the stencil arithmetic.  Waits are bounded (status bit 1 on expiry).
#include <cuda.h>
#include <cuda_runtime.h>

#include "yf_internal.h"

namespace yf {
namespace {

__device__ __forceinline__ int slab_s(int p, int N, int n, int lo, int hi)
{
    if (lo && p < n) return p;
    if (hi && p >= N - n) return n + p - (N - n);
    return -1;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mb_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mb_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mb_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mb_wait(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 26); ++it)
        if (mb_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma4(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int c,
                                     uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(c), "r"(bar)
        : "memory");
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T, int TX, int TY>
struct SkewLayout {
    static constexpr int XO = 16 / (int)sizeof(T);
    static constexpr int BX = TX + 2 * XO;
    static constexpr int WY = TY + 2;
    static constexpr int WN = BX * WY;
    static constexpr int WIN_BYTES = 3 * WN * (int)sizeof(T);
    static constexpr int WIN_PAD = (WIN_BYTES + 127) / 128 * 128;
    static constexpr int CLS_BYTES = 3 * TX * TY;
    static constexpr int CLS_PAD = (CLS_BYTES + 127) / 128 * 128;
    static constexpr int STAGE = 2 * WIN_PAD + CLS_PAD;
    static constexpr int NST = 4;
    static constexpr int SH_OFF = NST * STAGE;              // two new-H windows
    static constexpr int CT_OFF = SH_OFF + 2 * WIN_PAD;
    static constexpr int BAR_OFF = CT_OFF + (2 * kMaxClasses * (int)sizeof(T) + 127) / 128 * 128;
    static constexpr int BYTES = BAR_OFF + 64;
    static constexpr uint32_t TX_BYTES = 2 * WIN_BYTES + CLS_BYTES;
};

// CPML: psi_new = b psi_old + a d; returns d / kappa + psi_new
template <typename T>
__device__ __forceinline__ T cp(T d, T psi_old, T *w, const T *prof, int N1, int which, int p)
{
    const T v = prof[which * N1 + p] * psi_old + prof[(which + 1) * N1 + p] * d;
    if (w) *w = v;
    return d * prof[(which + 2) * N1 + p] + v;
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX *TY)
    k_yee_skew(FusedArgs<T> P, const __grid_constant__ CUtensorMap tmF,
               const __grid_constant__ CUtensorMap tmC, int *status)
{
    using Lay = SkewLayout<T, TX, TY>;
    using V2 = typename Vec2<T>::type;
    constexpr int XO = Lay::XO, BX = Lay::BX, WN = Lay::WN, NT = TX * TY, NST = Lay::NST;
    extern __shared__ __align__(128) unsigned char sm[];
    V2 *sC = reinterpret_cast<V2 *>(sm + Lay::CT_OFF);
    const uint32_t bar0 = smem_addr(sm + Lay::BAR_OFF);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = (blockIdx.x + P.tx0) * TX, j0 = (blockIdx.y + P.ty0) * TY;
    const int i = i0 + tx, j = j0 + ty;
    const int kb = P.z0 + blockIdx.z * P.kseg;
    if (kb > P.z1) return;
    const int ke = min(P.z1, kb + P.kseg - 1);
    const long plane = P.plane, npts = P.npts;
    const int px = P.px, NX1 = P.nx + 1, NY1 = P.ny + 1, NZ1 = P.nz + 1;
    const int n = P.n, L = P.L;

    if (smem_addr(sm) & 127u) {
        if (tid == 0) atomicOr(status, 4);
        return;
    }
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mb_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int q = tid; q < kMaxClasses; q += NT) sC[q] = V2{P.ctab[2 * q], P.ctab[2 * q + 1]};
    __syncthreads();

    auto issue = [&](int q, int s) {   // thread 0 only
        unsigned char *st = sm + s * Lay::STAGE;
        const uint32_t bar = bar0 + 8 * s;
        mb_expect_tx(bar, Lay::TX_BYTES);
        tma4(smem_addr(st), &tmF, i0 - XO, j0 - 1, q, 0, bar);
        tma4(smem_addr(st + Lay::WIN_PAD), &tmF, i0 - XO, j0 - 1, q, 3, bar);
        tma4(smem_addr(st + 2 * Lay::WIN_PAD), &tmC, i0, j0, q, 0, bar);
    };
    uint32_t phase = 0;
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // planes kb-1, kb, kb+1 now; the fourth stage gets kb+2 after the first iteration
        for (int q = kb - 1, s = 0; s < NST - 1 && q <= ke + 1; ++q, ++s) issue(q, s);
    }
    auto wait_stage = [&](int s) -> bool {
        bool ok = true;
        if (tid == 0) {
            ok = mb_wait(bar0 + 8 * s, (phase >> s) & 1u);
            phase ^= 1u << s;
        }
        return __syncthreads_and(ok);
    };
    if (!wait_stage(0)) {
        if (tid == 0) atomicOr(status, 2);
        return;
    }

    const bool live = i <= P.nx && j <= P.ny;
    const int sx = slab_s(i, P.nx, n, P.lo[0], P.hi[0]);
    const int sy = slab_s(j, P.ny, n, P.lo[1], P.hi[1]);
    const bool xy_slab = sx >= 0 || sy >= 0;
    const int wown = (ty + 1) * BX + (tx + XO);

    // halo H value of plane t owned by this thread (see yf_tma.cu for the assignment)
    constexpr int NHALO = 2 * TX + 2 * TY;
    static_assert(NHALO <= NT, "one halo value per thread");
    int h_comp = -1, h_w = 0, h_i = 0, h_j = 0, h_sx = -1, h_sy = -1;
    bool h_live = false;
    if (tid < NHALO) {
        if (tid < 2 * TX) {
            const int e = tid < TX ? tid : tid - TX;
            h_comp = tid < TX ? 0 : 2;
            h_w = e + XO;
            h_i = i0 + e;
            h_j = j0 - 1;
            h_live = j0 > 0 && h_i <= P.nx;
        } else {
            const int e = tid - 2 * TX;
            const int r = e < TY ? e : e - TY;
            h_comp = e < TY ? 1 : 2;
            h_w = (r + 1) * BX + (XO - 1);
            h_i = i0 - 1;
            h_j = j0 + r;
            h_live = i0 > 0 && h_j <= P.ny;
        }
        if (h_live) {
            h_sx = slab_s(h_i, P.nx, n, P.lo[0], P.hi[0]);
            h_sy = slab_s(h_j, P.ny, n, P.lo[1], P.hi[1]);
        }
    }

    // own H_x, H_y of planes t-1 (h1) and t-2 (h2)
    T hx1 = 0, hy1 = 0, hx2 = 0, hy2 = 0;
    // stages: plane t-1 -> s_m, t -> s_0, t+1 -> s_p
    int s_m = NST - 1, s_0 = 0, s_p = 1;
    for (int t = kb - 1; t <= ke + 1; ++t) {
        if (t + 1 <= ke + 1) {
            if (!wait_stage(s_p)) {
                if (tid == 0) atomicOr(status, 2);
                return;
            }
        }
        const int pe = t - 1;                        // plane of the E update
        const bool do_e = pe >= kb && live;
        const bool do_h = t <= ke && t >= 0;
        const int szh = do_h ? slab_s(t, P.nz, n, P.lo[2], P.hi[2]) : -1;
        const int sze = (pe >= kb) ? slab_s(pe, P.nz, n, P.lo[2], P.hi[2]) : -1;

        // ---- CPML auxiliaries of this iteration, fetched first ----
        T pe_y0 = 0, pe_z0 = 0, pe_z1 = 0, pe_x0 = 0, pe_x1 = 0, pe_y1 = 0;   // E: ex(y,z) ey(z,x) ez(x,y)
        T ph_y0 = 0, ph_z0 = 0, ph_z1 = 0, ph_x0 = 0, ph_x1 = 0, ph_y1 = 0;   // H: hx(y,z) hy(z,x) hz(x,y)
        const bool own_h = do_h && live;
        if (do_e && (xy_slab || sze >= 0)) {
            if (sy >= 0) {
                const long o = ((long)pe * L + sy) * px + i;
                pe_y0 = P.psiE[1][0][o];
                pe_y1 = P.psiE[1][1][o];
            }
            if (sze >= 0) {
                const long o = ((long)sze * NY1 + j) * px + i;
                pe_z0 = P.psiE[2][0][o];
                pe_z1 = P.psiE[2][1][o];
            }
            if (sx >= 0) {
                const long o = ((long)pe * NY1 + j) * L + sx;
                pe_x0 = P.psiE[0][0][o];
                pe_x1 = P.psiE[0][1][o];
            }
        }
        if (own_h && (xy_slab || szh >= 0)) {
            if (sy >= 0) {
                const long o = ((long)t * L + sy) * px + i;
                ph_y0 = P.psiHr[1][0][o];
                ph_y1 = P.psiHr[1][1][o];
            }
            if (szh >= 0) {
                const long o = ((long)szh * NY1 + j) * px + i;
                ph_z0 = P.psiHr[2][0][o];
                ph_z1 = P.psiHr[2][1][o];
            }
            if (sx >= 0) {
                const long o = ((long)t * NY1 + j) * L + sx;
                ph_x0 = P.psiHr[0][0][o];
                ph_x1 = P.psiHr[0][1][o];
            }
        }

        const unsigned char *stm = sm + s_m * Lay::STAGE;
        const unsigned char *st0 = sm + s_0 * Lay::STAGE;
        const unsigned char *stp = sm + s_p * Lay::STAGE;

        // ---- E^{n+1} on plane t - 1 ----
        if (do_e) {
            const T *shx = reinterpret_cast<const T *>(sm + Lay::SH_OFF + (pe & 1) * Lay::WIN_PAD);
            const T *shy = shx + WN, *shz = shy + WN;
            const T *eo = reinterpret_cast<const T *>(stm);   // E^n of plane t - 1
            const uint8_t *cl = stm + 2 * Lay::WIN_PAD;
            const long q = (long)pe * plane + (long)j * px + i;
            const int crow = ty * TX + tx;
            const T hxo = shx[wown], hyo = shy[wown], hzo = shz[wown];
            T exn = 0, eyn = 0, ezn = 0;
            int c = cl[crow];
            if (c) {   // E_x(i+1/2, j, pe) = Ca E_x + Cb (dHz/dy - dHy/dz)
                T d1 = (hzo - shz[wown - BX]) * P.rdy, d2 = (hyo - hy2) * P.rdz;
                if (sy >= 0) d1 = cp(d1, pe_y0, P.psiE[1][0] + ((long)pe * L + sy) * px + i, P.prof[1], NY1, 0, j);
                if (sze >= 0) d2 = cp(d2, pe_z0, P.psiE[2][0] + ((long)sze * NY1 + j) * px + i, P.prof[2], NZ1, 0, pe);
                const V2 k = sC[c];
                exn = k.x * eo[wown] + k.y * (d1 - d2);
            }
            c = cl[TX * TY + crow];
            if (c) {   // E_y(i, j+1/2, pe) = Ca E_y + Cb (dHx/dz - dHz/dx)
                T d1 = (hxo - hx2) * P.rdz, d2 = (hzo - shz[wown - 1]) * P.rdx;
                if (sze >= 0) d1 = cp(d1, pe_z1, P.psiE[2][1] + ((long)sze * NY1 + j) * px + i, P.prof[2], NZ1, 0, pe);
                if (sx >= 0) d2 = cp(d2, pe_x0, P.psiE[0][0] + ((long)pe * NY1 + j) * L + sx, P.prof[0], NX1, 0, i);
                const V2 k = sC[c];
                eyn = k.x * eo[WN + wown] + k.y * (d1 - d2);
            }
            c = cl[2 * TX * TY + crow];
            if (c) {   // E_z(i, j, pe+1/2) = Ca E_z + Cb (dHy/dx - dHx/dy)
                T d1 = (hyo - shy[wown - 1]) * P.rdx, d2 = (hxo - shx[wown - BX]) * P.rdy;
                if (sx >= 0) d1 = cp(d1, pe_x1, P.psiE[0][1] + ((long)pe * NY1 + j) * L + sx, P.prof[0], NX1, 0, i);
                if (sy >= 0) d2 = cp(d2, pe_y1, P.psiE[1][1] + ((long)pe * L + sy) * px + i, P.prof[1], NY1, 0, j);
                const V2 k = sC[c];
                ezn = k.x * eo[2 * WN + wown] + k.y * (d1 - d2);
            }
            P.B[q] = exn;
            P.B[npts + q] = eyn;
            P.B[2 * npts + q] = ezn;
        }

        // ---- H^{n+1/2} on plane t ----
        if (do_h) {
            const T *ex0 = reinterpret_cast<const T *>(st0), *ey0 = ex0 + WN, *ez0 = ey0 + WN;
            const T *hox = reinterpret_cast<const T *>(st0 + Lay::WIN_PAD), *hoy = hox + WN, *hoz = hoy + WN;
            const T *ex1 = reinterpret_cast<const T *>(stp), *ey1 = ex1 + WN;
            T *snx = reinterpret_cast<T *>(sm + Lay::SH_OFF + (t & 1) * Lay::WIN_PAD);
            T *sny = snx + WN, *snz = sny + WN;
            const bool warm = t < kb;
            T hx = 0, hy = 0, hz = 0;
            if (live) {
                const int w = wown;
                const bool vx = !warm && j < P.ny && t < P.nz;
                const bool vy = !warm && i < P.nx && t < P.nz;
                const bool vz = !warm && i < P.nx && j < P.ny;
                T d1 = (ez0[w + BX] - ez0[w]) * P.rdy, d2 = (ey1[w] - ey0[w]) * P.rdz;
                if (sy >= 0) d1 = cp(d1, ph_y0, vx ? P.psiHw[1][0] + ((long)t * L + sy) * px + i : (T *)nullptr, P.prof[1], NY1, 3, j);
                if (szh >= 0) d2 = cp(d2, ph_z0, vx ? P.psiHw[2][0] + ((long)szh * NY1 + j) * px + i : (T *)nullptr, P.prof[2], NZ1, 3, t);
                hx = hox[w] - P.db * (d1 - d2);
                d1 = (ex1[w] - ex0[w]) * P.rdz;
                d2 = (ez0[w + 1] - ez0[w]) * P.rdx;
                if (szh >= 0) d1 = cp(d1, ph_z1, vy ? P.psiHw[2][1] + ((long)szh * NY1 + j) * px + i : (T *)nullptr, P.prof[2], NZ1, 3, t);
                if (sx >= 0) d2 = cp(d2, ph_x0, vy ? P.psiHw[0][0] + ((long)t * NY1 + j) * L + sx : (T *)nullptr, P.prof[0], NX1, 3, i);
                hy = hoy[w] - P.db * (d1 - d2);
                if (!warm) {
                    d1 = (ey0[w + 1] - ey0[w]) * P.rdx;
                    d2 = (ex0[w + BX] - ex0[w]) * P.rdy;
                    if (sx >= 0) d1 = cp(d1, ph_x1, vz ? P.psiHw[0][1] + ((long)t * NY1 + j) * L + sx : (T *)nullptr, P.prof[0], NX1, 3, i);
                    if (sy >= 0) d2 = cp(d2, ph_y1, vz ? P.psiHw[1][1] + ((long)t * L + sy) * px + i : (T *)nullptr, P.prof[1], NY1, 3, j);
                    hz = hoz[w] - P.db * (d1 - d2);
                    const long q = (long)t * plane + (long)j * px + i;
                    if (vx) P.B[3 * npts + q] = hx;
                    if (vy) P.B[4 * npts + q] = hy;
                    if (vz) P.B[5 * npts + q] = hz;
                }
            }
            if (!warm) {
                snx[wown] = hx;
                sny[wown] = hy;
                snz[wown] = hz;
                if (h_comp >= 0) {
                    T v = 0;
                    if (h_live) {
                        const int w = h_w;
                        if (h_comp == 0) {
                            T d1 = (ez0[w + BX] - ez0[w]) * P.rdy, d2 = (ey1[w] - ey0[w]) * P.rdz;
                            if (h_sy >= 0) d1 = cp(d1, P.psiHr[1][0][((long)t * L + h_sy) * px + h_i], (T *)nullptr, P.prof[1], NY1, 3, h_j);
                            if (szh >= 0) d2 = cp(d2, P.psiHr[2][0][((long)szh * NY1 + h_j) * px + h_i], (T *)nullptr, P.prof[2], NZ1, 3, t);
                            v = hox[w] - P.db * (d1 - d2);
                        } else if (h_comp == 1) {
                            T d1 = (ex1[w] - ex0[w]) * P.rdz, d2 = (ez0[w + 1] - ez0[w]) * P.rdx;
                            if (szh >= 0) d1 = cp(d1, P.psiHr[2][1][((long)szh * NY1 + h_j) * px + h_i], (T *)nullptr, P.prof[2], NZ1, 3, t);
                            if (h_sx >= 0) d2 = cp(d2, P.psiHr[0][0][((long)t * NY1 + h_j) * L + h_sx], (T *)nullptr, P.prof[0], NX1, 3, h_i);
                            v = hoy[w] - P.db * (d1 - d2);
                        } else {
                            T d1 = (ey0[w + 1] - ey0[w]) * P.rdx, d2 = (ex0[w + BX] - ex0[w]) * P.rdy;
                            if (h_sx >= 0) d1 = cp(d1, P.psiHr[0][1][((long)t * NY1 + h_j) * L + h_sx], (T *)nullptr, P.prof[0], NX1, 3, h_i);
                            if (h_sy >= 0) d2 = cp(d2, P.psiHr[1][1][((long)t * L + h_sy) * px + h_i], (T *)nullptr, P.prof[1], NY1, 3, h_j);
                            v = hoz[w] - P.db * (d1 - d2);
                        }
                    }
                    if (h_comp == 0) snx[h_w] = v;
                    else if (h_comp == 1) sny[h_w] = v;
                    else snz[h_w] = v;
                }
            }
            hx2 = hx1;
            hy2 = hy1;
            hx1 = hx;
            hy1 = hy;
        } else {
            hx2 = hx1;
            hy2 = hy1;
            hx1 = 0;
            hy1 = 0;
        }

        __syncthreads();
        // stage s_m (plane t - 1) is no longer needed: refill it with plane t + 3
        if (tid == 0 && t + 3 <= ke + 1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(t + 3, s_m);
        }
        s_m = s_0;
        s_0 = s_p;
        s_p = s_p == NST - 1 ? 0 : s_p + 1;
    }
}

template <typename T, int TX, int TY>
cudaError_t launch_skew_t(const FusedArgs<T> &a, const CUtensorMap &tmF, const CUtensorMap &tmC,
                          int *status, cudaStream_t s)
{
    using Lay = SkewLayout<T, TX, TY>;
    dim3 blk(TX, TY), grd((a.nx + 1 + TX - 1) / TX, (a.ny + 1 + TY - 1) / TY,
                          (a.nz + 1 + a.kseg - 1) / a.kseg);
    k_yee_skew<T, TX, TY><<<grd, blk, Lay::BYTES, s>>>(a, tmF, tmC, status);
    return cudaGetLastError();
}

template <typename T, int TX, int TY>
cudaError_t prep_skew()
{
    return cudaFuncSetAttribute(k_yee_skew<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SkewLayout<T, TX, TY>::BYTES);
}

}  // namespace

cudaError_t skew_prepare()
{
    cudaError_t e;
    if ((e = prep_skew<float, 32, 4>()) != cudaSuccess) return e;
    if ((e = prep_skew<float, 32, 8>()) != cudaSuccess) return e;
    if ((e = prep_skew<float, 32, 16>()) != cudaSuccess) return e;
    if ((e = prep_skew<double, 32, 4>()) != cudaSuccess) return e;
    if ((e = prep_skew<double, 32, 8>()) != cudaSuccess) return e;
    return prep_skew<double, 32, 16>();
}

template <typename T>
cudaError_t launch_skew(const FusedArgs<T> &a, const CUtensorMap &tmF, const CUtensorMap &tmC,
                        int tile_y, int *status, cudaStream_t s)
{
    switch (tile_y) {
    case 4: return launch_skew_t<T, 32, 4>(a, tmF, tmC, status, s);
    case 16: return launch_skew_t<T, 32, 16>(a, tmF, tmC, status, s);
    default: return launch_skew_t<T, 32, 8>(a, tmF, tmC, status, s);
    }
}

template cudaError_t launch_skew<float>(const FusedArgs<float> &, const CUtensorMap &,
                                        const CUtensorMap &, int, int *, cudaStream_t);
template cudaError_t launch_skew<double>(const FusedArgs<double> &, const CUtensorMap &,
                                         const CUtensorMap &, int, int *, cudaStream_t);

}  // namespace yf
