// Fused Yee step with TMA-staged planes (variant 2).
//
// Same update and same z-march as k_yee_fused (yf_fused.cu): buffer A -> buffer B, halo H
// recomputed, H^{n+1/2} of plane p-1 kept in registers.  The difference is how plane data
// reaches shared memory: one elected thread issues tensor-memory-accelerator loads
// (cp.async.bulk.tensor, 4-D tensor maps over [component][z][y][x]) of
//   - the E^n window   (3 components, x in [i0 - XO, i0 + TX + XO), y in [j0 - 1, j0 + TY]),
//   - the H^{n-1/2} window (same box, components 3..5),
//   - the three uint8 edge-class tiles (x in [i0, i0 + TX), y in [j0, j0 + TY)),
// of plane q into stage q mod 3, completing on that stage's mbarrier.  Planes are issued
// three ahead of the one being computed, so HBM latency overlaps the arithmetic of the two
// planes before.  The x origin i0 - XO is a multiple of 16 bytes (XO = 16 / sizeof(T)); nodes
// outside the grid arrive as zeros (TMA out-of-bounds fill).  Every mbarrier wait is bounded:
// on expiry the block sets bit 1 of the status word and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include "yf_internal.h"

namespace yf {
namespace {

__device__ __forceinline__ int slab_i(int p, int N, int n, int lo, int hi)
{
    if (lo && p < n) return p;
    if (hi && p >= N - n) return n + p - (N - n);
    return -1;
}

template <typename T>
__device__ __forceinline__ T cpml_x(T d, const T *r, T *w, const T *prof, int N1, int which, int p)
{
    const T b = prof[(which + 0) * N1 + p];
    const T a = prof[(which + 1) * N1 + p];
    const T rk = prof[(which + 2) * N1 + p];
    const T v = b * (*r) + a * d;
    if (w) *w = v;
    return d * rk + v;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
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

// bounded wait: about 2^26 polls (seconds) before giving up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 26); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            int z, int c, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(c), "r"(bar)
        : "memory");
}


template <typename T, int TX, int TY>
struct TmaLayout {
    static constexpr int XO = 16 / (int)sizeof(T);   // x halo rounded to 16 bytes
    static constexpr int BX = TX + 2 * XO;           // window width
    static constexpr int WY = TY + 2;                // window height
    static constexpr int WN = BX * WY;               // nodes per window plane
    static constexpr int WIN_BYTES = 3 * WN * (int)sizeof(T);
    static constexpr int WIN_PAD = (WIN_BYTES + 127) / 128 * 128;
    static constexpr int CLS_BYTES = 3 * TX * TY;
    static constexpr int CLS_PAD = (CLS_BYTES + 127) / 128 * 128;
    static constexpr int STAGE = 2 * WIN_PAD + CLS_PAD;   // E window, H window, classes
    static constexpr int NST = 3;
    static constexpr int SH_OFF = NST * STAGE;            // new H window
    static constexpr int CT_OFF = SH_OFF + WIN_PAD;       // (Ca, Cb) pairs
    static constexpr int BAR_OFF = CT_OFF + (2 * kMaxClasses * (int)sizeof(T) + 127) / 128 * 128;
    static constexpr int BYTES = BAR_OFF + 64;
    static constexpr uint32_t TX_BYTES = 2 * WIN_BYTES + CLS_BYTES;
};

template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// CPML-corrected derivative of an H component without the auxiliary write (halo nodes and
// the warm-up plane recompute values whose owner writes the auxiliaries).
template <typename T>
__device__ __forceinline__ T read_term(T d, const T *psi, long o, const T *prof, int N1, int p)
{
    return cpml_x<T>(d, psi + o, (T *)nullptr, prof, N1, 3, p);
}

// Block: TX x TYT threads; thread (tx, ty) owns node column i = i0 + tx and the CY rows
// j = j0 + ty*CY + r (r < CY) of a TX x (TYT*CY) tile.  Rows of one thread are contiguous, so
// the y neighbours of its E and H values come from registers, E^n read for the H update is
// reused by the E update, and the loop overhead of a plane is paid once per CY nodes.
template <typename T, int TX, int TYT, int CY, bool HP>
__global__ void __launch_bounds__(TX *TYT)
    k_yee_tma(FusedArgs<T> P, const __grid_constant__ CUtensorMap tmF,
              const __grid_constant__ CUtensorMap tmC, int *status)
{
    constexpr int TY = TYT * CY;
    using Lay = TmaLayout<T, TX, TY>;
    using P2 = typename Pair<T>::type;
    constexpr int XO = Lay::XO, BX = Lay::BX, WN = Lay::WN, NT = TX * TYT;
    extern __shared__ __align__(128) unsigned char sm[];
    T *sHn = reinterpret_cast<T *>(sm + Lay::SH_OFF);
    P2 *sC = reinterpret_cast<P2 *>(sm + Lay::CT_OFF);
    const uint32_t bar0 = smem_u32(sm + Lay::BAR_OFF);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = (blockIdx.x + P.tx0) * TX, j0 = (blockIdx.y + P.ty0) * TY;
    const int i = i0 + tx, jb = j0 + ty * CY;
    const int kb = P.z0 + blockIdx.z * P.kseg;
    if (kb > P.z1) return;
    const int ke = min(P.z1, kb + P.kseg - 1);
    const long plane = P.plane, npts = P.npts;
    const int px = P.px, NX1 = P.nx + 1, NY1 = P.ny + 1, NZ1 = P.nz + 1;
    const int n = P.n, L = P.L;

    // TMA writes need 128-byte aligned shared destinations
    if (smem_u32(sm) & 127u) {
        if (tid == 0) atomicOr(status, 4);
        return;
    }
    if (tid == 0) {
        for (int s = 0; s < Lay::NST; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int q = tid; q < kMaxClasses; q += NT) sC[q] = P2{P.ctab[2 * q], P.ctab[2 * q + 1]};
    __syncthreads();

    // plane q lives in stage (q - kb + 1) mod 3; thread 0 tracks the parity of each stage's
    // next completion in `phase` (bit s)
    auto issue = [&](int q, int s) {   // thread 0 only
        unsigned char *st = sm + s * Lay::STAGE;
        const uint32_t bar = bar0 + 8 * s;
        mbar_expect_tx(bar, Lay::TX_BYTES);
        tma_load_4d(smem_u32(st), &tmF, i0 - XO, j0 - 1, q, 0, bar);
        tma_load_4d(smem_u32(st + Lay::WIN_PAD), &tmF, i0 - XO, j0 - 1, q, 3, bar);
        tma_load_4d(smem_u32(st + 2 * Lay::WIN_PAD), &tmC, i0, j0, q, 0, bar);
    };
    uint32_t phase = 0;
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int q = kb - 1, s = 0; q <= kb + 1 && q <= ke + 1; ++q, ++s) issue(q, s);
    }
    // one thread polls the stage barrier; the others sleep in the block barrier
    auto wait_stage = [&](int s) -> bool {
        bool ok = true;
        if (tid == 0) {
            ok = mbar_wait(bar0 + 8 * s, (phase >> s) & 1u);
            phase ^= 1u << s;
        }
        return __syncthreads_and(ok);
    };
    if (!wait_stage(0)) {
        if (tid == 0) atomicOr(status, 2);
        return;
    }

    // per-thread constants
    const bool col_live = i <= P.nx;
    const int sx = slab_i(i, P.nx, n, P.lo[0], P.hi[0]);
    int sy[CY];
    bool rlive[CY];
#pragma unroll
    for (int r = 0; r < CY; ++r) {
        sy[r] = slab_i(jb + r, P.ny, n, P.lo[1], P.hi[1]);
        rlive[r] = col_live && jb + r <= P.ny;
    }
    const int w0 = (ty * CY + 1) * BX + (tx + XO);   // window index of row r: w0 + r * BX

    // halo value owned by this thread (threads 0 .. 2TX+2TY-1): the row j0-1 needs H_x and
    // H_z for i0 <= i < i0+TX, the column i0-1 needs H_y and H_z for j0 <= j < j0+TY.
    // h_comp: 0 H_x, 1 H_y, 2 H_z, -1 none; h_live false stores a zero (outside the grid)
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
            h_sx = slab_i(h_i, P.nx, n, P.lo[0], P.hi[0]);
            h_sy = slab_i(h_j, P.ny, n, P.lo[1], P.hi[1]);
        }
    }

    T hx_prev[CY], hy_prev[CY];
#pragma unroll
    for (int r = 0; r < CY; ++r) hx_prev[r] = hy_prev[r] = 0;
    int sp = 0, sn = 1;   // stages of planes p and p + 1
    for (int p = kb - 1; p <= ke; ++p) {
        // plane p + 1 must have landed (its E is the upper neighbour of plane p's H)
        if (!wait_stage(sn)) {
            if (tid == 0) atomicOr(status, 2);
            return;
        }
        const unsigned char *stp = sm + sp * Lay::STAGE;
        const unsigned char *stn = sm + sn * Lay::STAGE;
        const T *ex0 = reinterpret_cast<const T *>(stp), *ey0 = ex0 + WN, *ez0 = ey0 + WN;
        const T *hox = reinterpret_cast<const T *>(stp + Lay::WIN_PAD), *hoy = hox + WN, *hoz = hoy + WN;
        const uint8_t *cl = stp + 2 * Lay::WIN_PAD;
        const T *ex1 = reinterpret_cast<const T *>(stn), *ey1 = ex1 + WN;
        const bool pin = p >= 0;
        const int sz = pin ? slab_i(p, P.nz, n, P.lo[2], P.hi[2]) : -1;

        // E^n of this thread's rows (plus the row above for the y differences)
        T exv[CY + 1], ezv[CY + 1], eyv[CY], eyx[CY], ezx[CY], ey1v[CY], ex1v[CY];
#pragma unroll
        for (int r = 0; r <= CY; ++r) {
            exv[r] = ex0[w0 + r * BX];
            ezv[r] = ez0[w0 + r * BX];
        }
#pragma unroll
        for (int r = 0; r < CY; ++r) {
            const int w = w0 + r * BX;
            eyv[r] = ey0[w];
            eyx[r] = ey0[w + 1];
            ezx[r] = ez0[w + 1];
            ey1v[r] = ey1[w];
            ex1v[r] = ex1[w];
        }

        if (p < kb) {
            // warm-up plane kb - 1: own H_x, H_y (the E update of plane kb needs them)
            if (pin && p < P.nz) {
#pragma unroll
                for (int r = 0; r < CY; ++r) {
                    const int w = w0 + r * BX, j = jb + r;
                    T d1 = (ezv[r + 1] - ezv[r]) * P.rdy, d2 = (ey1v[r] - eyv[r]) * P.rdz;
                    if (HP && sy[r] >= 0) d1 = read_term(d1, P.psiHr[1][0], ((long)p * L + sy[r]) * px + i, P.prof[1], NY1, j);
                    if (HP && sz >= 0) d2 = read_term(d2, P.psiHr[2][0], ((long)sz * NY1 + j) * px + i, P.prof[2], NZ1, p);
                    hx_prev[r] = hox[w] - P.db * (d1 - d2);
                    d1 = (ex1v[r] - exv[r]) * P.rdz;
                    d2 = (ezx[r] - ezv[r]) * P.rdx;
                    if (HP && sz >= 0) d1 = read_term(d1, P.psiHr[2][1], ((long)sz * NY1 + j) * px + i, P.prof[2], NZ1, p);
                    if (HP && sx >= 0) d2 = read_term(d2, P.psiHr[0][0], ((long)p * NY1 + j) * L + sx, P.prof[0], NX1, i);
                    hy_prev[r] = hoy[w] - P.db * (d1 - d2);
                }
            }
        } else {
            const long qb = (long)p * plane + (long)jb * px + i;
            T hx[CY], hy[CY], hz[CY];
#pragma unroll
            for (int r = 0; r < CY; ++r) {
                const int w = w0 + r * BX, j = jb + r;
                const bool vx = rlive[r] && j < P.ny && p < P.nz;
                const bool vy = rlive[r] && i < P.nx && p < P.nz;
                const bool vz = rlive[r] && i < P.nx && j < P.ny;
                // H_x(i, j+1/2, p+1/2) -= dt/mu0 (dEz/dy - dEy/dz)
                T d1 = (ezv[r + 1] - ezv[r]) * P.rdy, d2 = (ey1v[r] - eyv[r]) * P.rdz;
                if (HP && sy[r] >= 0) {
                    const long o = ((long)p * L + sy[r]) * px + i;
                    d1 = cpml_x(d1, P.psiHr[1][0] + o, vx ? P.psiHw[1][0] + o : (T *)nullptr, P.prof[1], NY1, 3, j);
                }
                if (HP && sz >= 0) {
                    const long o = ((long)sz * NY1 + j) * px + i;
                    d2 = cpml_x(d2, P.psiHr[2][0] + o, vx ? P.psiHw[2][0] + o : (T *)nullptr, P.prof[2], NZ1, 3, p);
                }
                hx[r] = hox[w] - P.db * (d1 - d2);
                // H_y(i+1/2, j, p+1/2) -= dt/mu0 (dEx/dz - dEz/dx)
                d1 = (ex1v[r] - exv[r]) * P.rdz;
                d2 = (ezx[r] - ezv[r]) * P.rdx;
                if (HP && sz >= 0) {
                    const long o = ((long)sz * NY1 + j) * px + i;
                    d1 = cpml_x(d1, P.psiHr[2][1] + o, vy ? P.psiHw[2][1] + o : (T *)nullptr, P.prof[2], NZ1, 3, p);
                }
                if (HP && sx >= 0) {
                    const long o = ((long)p * NY1 + j) * L + sx;
                    d2 = cpml_x(d2, P.psiHr[0][0] + o, vy ? P.psiHw[0][0] + o : (T *)nullptr, P.prof[0], NX1, 3, i);
                }
                hy[r] = hoy[w] - P.db * (d1 - d2);
                // H_z(i+1/2, j+1/2, p) -= dt/mu0 (dEy/dx - dEx/dy)
                d1 = (eyx[r] - eyv[r]) * P.rdx;
                d2 = (exv[r + 1] - exv[r]) * P.rdy;
                if (HP && sx >= 0) {
                    const long o = ((long)p * NY1 + j) * L + sx;
                    d1 = cpml_x(d1, P.psiHr[0][1] + o, vz ? P.psiHw[0][1] + o : (T *)nullptr, P.prof[0], NX1, 3, i);
                }
                if (HP && sy[r] >= 0) {
                    const long o = ((long)p * L + sy[r]) * px + i;
                    d2 = cpml_x(d2, P.psiHr[1][1] + o, vz ? P.psiHw[1][1] + o : (T *)nullptr, P.prof[1], NY1, 3, j);
                }
                hz[r] = hoz[w] - P.db * (d1 - d2);
                sHn[w] = hx[r];
                sHn[WN + w] = hy[r];
                sHn[2 * WN + w] = hz[r];
                const long q = qb + (long)r * px;
                if (vx) P.B[3 * npts + q] = hx[r];
                if (vy) P.B[4 * npts + q] = hy[r];
                if (vz) P.B[5 * npts + q] = hz[r];
            }
            if (h_comp >= 0) {   // one halo H value per thread of the first warps
                T v = 0;
                if (h_live) {
                    const int w = h_w;
                    if (h_comp == 0) {
                        T d1 = (ez0[w + BX] - ez0[w]) * P.rdy, d2 = (ey1[w] - ey0[w]) * P.rdz;
                        if (HP && h_sy >= 0) d1 = read_term(d1, P.psiHr[1][0], ((long)p * L + h_sy) * px + h_i, P.prof[1], NY1, h_j);
                        if (HP && sz >= 0) d2 = read_term(d2, P.psiHr[2][0], ((long)sz * NY1 + h_j) * px + h_i, P.prof[2], NZ1, p);
                        v = hox[w] - P.db * (d1 - d2);
                    } else if (h_comp == 1) {
                        T d1 = (ex1[w] - ex0[w]) * P.rdz, d2 = (ez0[w + 1] - ez0[w]) * P.rdx;
                        if (HP && sz >= 0) d1 = read_term(d1, P.psiHr[2][1], ((long)sz * NY1 + h_j) * px + h_i, P.prof[2], NZ1, p);
                        if (HP && h_sx >= 0) d2 = read_term(d2, P.psiHr[0][0], ((long)p * NY1 + h_j) * L + h_sx, P.prof[0], NX1, h_i);
                        v = hoy[w] - P.db * (d1 - d2);
                    } else {
                        T d1 = (ey0[w + 1] - ey0[w]) * P.rdx, d2 = (ex0[w + BX] - ex0[w]) * P.rdy;
                        if (HP && h_sx >= 0) d1 = read_term(d1, P.psiHr[0][1], ((long)p * NY1 + h_j) * L + h_sx, P.prof[0], NX1, h_i);
                        if (HP && h_sy >= 0) d2 = read_term(d2, P.psiHr[1][1], ((long)p * L + h_sy) * px + h_i, P.prof[1], NY1, h_j);
                        v = hoz[w] - P.db * (d1 - d2);
                    }
                }
                sHn[h_comp * WN + h_w] = v;
            }
            __syncthreads();

            const T *shx = sHn, *shy = sHn + WN, *shz = sHn + 2 * WN;
            T hz_up = shz[w0 - BX], hx_up = shx[w0 - BX];
#pragma unroll
            for (int r = 0; r < CY; ++r) {
                const int w = w0 + r * BX, j = jb + r;
                const int crow = (ty * CY + r) * TX + tx;
                T exn = 0, eyn = 0, ezn = 0;
                int c = cl[crow];
                if (c) {   // E_x(i+1/2, j, p) = Ca E_x + Cb (dHz/dy - dHy/dz)
                    T d1 = (hz[r] - hz_up) * P.rdy, d2 = (hy[r] - hy_prev[r]) * P.rdz;
                    if (HP && sy[r] >= 0) {
                        T *o = P.psiE[1][0] + ((long)p * L + sy[r]) * px + i;
                        d1 = cpml_x(d1, o, o, P.prof[1], NY1, 0, j);
                    }
                    if (HP && sz >= 0) {
                        T *o = P.psiE[2][0] + ((long)sz * NY1 + j) * px + i;
                        d2 = cpml_x(d2, o, o, P.prof[2], NZ1, 0, p);
                    }
                    const P2 k = sC[c];
                    exn = k.x * exv[r] + k.y * (d1 - d2);
                }
                c = cl[TX * TY + crow];
                if (c) {   // E_y(i, j+1/2, p) = Ca E_y + Cb (dHx/dz - dHz/dx)
                    T d1 = (hx[r] - hx_prev[r]) * P.rdz, d2 = (hz[r] - shz[w - 1]) * P.rdx;
                    if (HP && sz >= 0) {
                        T *o = P.psiE[2][1] + ((long)sz * NY1 + j) * px + i;
                        d1 = cpml_x(d1, o, o, P.prof[2], NZ1, 0, p);
                    }
                    if (HP && sx >= 0) {
                        T *o = P.psiE[0][0] + ((long)p * NY1 + j) * L + sx;
                        d2 = cpml_x(d2, o, o, P.prof[0], NX1, 0, i);
                    }
                    const P2 k = sC[c];
                    eyn = k.x * eyv[r] + k.y * (d1 - d2);
                }
                c = cl[2 * TX * TY + crow];
                if (c) {   // E_z(i, j, p+1/2) = Ca E_z + Cb (dHy/dx - dHx/dy)
                    T d1 = (hy[r] - shy[w - 1]) * P.rdx, d2 = (hx[r] - hx_up) * P.rdy;
                    if (HP && sx >= 0) {
                        T *o = P.psiE[0][1] + ((long)p * NY1 + j) * L + sx;
                        d1 = cpml_x(d1, o, o, P.prof[0], NX1, 0, i);
                    }
                    if (HP && sy[r] >= 0) {
                        T *o = P.psiE[1][1] + ((long)p * L + sy[r]) * px + i;
                        d2 = cpml_x(d2, o, o, P.prof[1], NY1, 0, j);
                    }
                    const P2 k = sC[c];
                    ezn = k.x * ezv[r] + k.y * (d1 - d2);
                }
                if (rlive[r]) {
                    const long q = qb + (long)r * px;
                    P.B[q] = exn;
                    P.B[npts + q] = eyn;
                    P.B[2 * npts + q] = ezn;
                }
                hz_up = hz[r];
                hx_up = hx[r];
                hx_prev[r] = hx[r];
                hy_prev[r] = hy[r];
            }
        }
        // every thread is done with stage sp: refill it with plane p + 3
        __syncthreads();
        if (tid == 0 && p + 3 <= ke + 1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(p + 3, sp);
        }
        sp = sn;
        sn = sn == Lay::NST - 1 ? 0 : sn + 1;
    }
}

// one launch over tiles [tx0, tx1) x [ty0, ty1) and planes z0..z1
template <typename T, int TX, int TYT, int CY, bool HP>
cudaError_t launch_box(FusedArgs<T> a, const CUtensorMap &tmF, const CUtensorMap &tmC, int *status,
                       cudaStream_t s, int tx0, int tx1, int ty0, int ty1, int z0, int z1)
{
    using Lay = TmaLayout<T, TX, TYT * CY>;
    if (tx1 <= tx0 || ty1 <= ty0 || z1 < z0) return cudaSuccess;
    a.tx0 = tx0; a.ty0 = ty0; a.z0 = z0; a.z1 = z1;
    dim3 blk(TX, TYT), grd(tx1 - tx0, ty1 - ty0, (z1 - z0 + 1 + a.kseg - 1) / a.kseg);
    k_yee_tma<T, TX, TYT, CY, HP><<<grd, blk, Lay::BYTES, s>>>(a, tmF, tmC, status);
    return cudaGetLastError();
}

// The instantiation without CPML code (about half the registers) covers the box of tiles and
// planes whose nodes, halo nodes and warm-up plane touch no absorbing slab; the CPML
// instantiation covers the frame around it (at most six boxes).  Every launch reads buffer A
// and writes a disjoint part of buffer B.
template <typename T, int TX, int TYT, int CY>
cudaError_t launch_tma_t(const FusedArgs<T> &a, const CUtensorMap &tmF, const CUtensorMap &tmC,
                         int *status, cudaStream_t s, const SideStream *side)
{
    constexpr int TY = TYT * CY;
    const int ntx = (a.nx + 1 + TX - 1) / TX, nty = (a.ny + 1 + TY - 1) / TY, nz = a.nz, n = a.n;
    const bool hp = n > 0 && (a.lo[0] || a.hi[0] || a.lo[1] || a.hi[1] || a.lo[2] || a.hi[2]);
    if (!hp) return launch_box<T, TX, TYT, CY, false>(a, tmF, tmC, status, s, 0, ntx, 0, nty, 0, nz);
    // interior: halo column i0-1 >= n and last node i0+TX-1 < nx-n (same in y); planes from
    // the warm-up plane on stay outside the z slabs
    auto lo_tile = [](int on, int n_, int tile) { return on ? (n_ + 1 + tile - 1) / tile : 0; };
    auto hi_tile = [](int on, int N, int n_, int tile, int count) {
        if (!on) return count;
        const int lim = N - n_ - tile;   // largest i0 with i0 + tile - 1 < N - n
        return lim < 0 ? 0 : lim / tile + 1;
    };
    const int txa = lo_tile(a.lo[0], n, TX), txb = min(ntx, hi_tile(a.hi[0], a.nx, n, TX, ntx));
    const int tya = lo_tile(a.lo[1], n, TY), tyb = min(nty, hi_tile(a.hi[1], a.ny, n, TY, nty));
    const int za = a.lo[2] ? n + 1 : 0, zb = a.hi[2] ? nz - n - 1 : nz;
    if (txa >= txb || tya >= tyb || za > zb)
        return launch_box<T, TX, TYT, CY, true>(a, tmF, tmC, status, s, 0, ntx, 0, nty, 0, nz);
    // the frame (latency-bound CPML work) runs on a side stream next to the interior
    // (bandwidth-bound), joined back before the step's epilogue
    cudaError_t e;
    cudaStream_t fs = s;
    if (side && side->stream) {
        if ((e = cudaEventRecord(side->fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side->stream, side->fork, 0)) != cudaSuccess) return e;
        fs = side->stream;
    }
    if ((e = launch_box<T, TX, TYT, CY, true>(a, tmF, tmC, status, fs, 0, ntx, 0, nty, zb + 1, nz)) != cudaSuccess) return e;
    if ((e = launch_box<T, TX, TYT, CY, true>(a, tmF, tmC, status, fs, 0, txa, 0, nty, za, zb)) != cudaSuccess) return e;
    if ((e = launch_box<T, TX, TYT, CY, true>(a, tmF, tmC, status, fs, txb, ntx, 0, nty, za, zb)) != cudaSuccess) return e;
    if ((e = launch_box<T, TX, TYT, CY, true>(a, tmF, tmC, status, fs, txa, txb, 0, tya, za, zb)) != cudaSuccess) return e;
    if ((e = launch_box<T, TX, TYT, CY, true>(a, tmF, tmC, status, fs, txa, txb, tyb, nty, za, zb)) != cudaSuccess) return e;
    if ((e = launch_box<T, TX, TYT, CY, true>(a, tmF, tmC, status, fs, 0, ntx, 0, nty, 0, za - 1)) != cudaSuccess) return e;
    if ((e = launch_box<T, TX, TYT, CY, false>(a, tmF, tmC, status, s, txa, txb, tya, tyb, za, zb)) != cudaSuccess) return e;
    if (fs != s) {
        if ((e = cudaEventRecord(side->join, fs)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, side->join, 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T, int TX, int TYT, int CY>
cudaError_t prepare_t()
{
    cudaError_t e = cudaFuncSetAttribute(k_yee_tma<T, TX, TYT, CY, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TmaLayout<T, TX, TYT * CY>::BYTES);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_yee_tma<T, TX, TYT, CY, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TmaLayout<T, TX, TYT * CY>::BYTES);
}

}  // namespace

template <typename T>
int tma_box_x(int tile_x) { return tile_x + 2 * (16 / (int)sizeof(T)); }

// shared-memory opt-in of every instantiation; call outside stream capture
cudaError_t tma_prepare()
{
    cudaError_t e;
    if ((e = prepare_t<float, 32, 4, 1>()) != cudaSuccess) return e;
    if ((e = prepare_t<float, 32, 8, 1>()) != cudaSuccess) return e;
    if ((e = prepare_t<float, 32, 8, 2>()) != cudaSuccess) return e;
    if ((e = prepare_t<double, 32, 4, 1>()) != cudaSuccess) return e;
    if ((e = prepare_t<double, 32, 8, 1>()) != cudaSuccess) return e;
    return prepare_t<double, 32, 8, 2>();
}

// tile_y = rows per block: 4 -> 4 threads x 1 row, 8 -> 8 x 1, 16 -> 8 x 2
template <typename T>
cudaError_t launch_tma(const FusedArgs<T> &a, const CUtensorMap &tmF, const CUtensorMap &tmC,
                       int tile_y, int *status, cudaStream_t s, const SideStream *side)
{
    switch (tile_y) {
    case 4: return launch_tma_t<T, 32, 4, 1>(a, tmF, tmC, status, s, side);
    case 16: return launch_tma_t<T, 32, 8, 2>(a, tmF, tmC, status, s, side);
    default: return launch_tma_t<T, 32, 8, 1>(a, tmF, tmC, status, s, side);
    }
}

template int tma_box_x<float>(int);
template int tma_box_x<double>(int);
template cudaError_t launch_tma<float>(const FusedArgs<float> &, const CUtensorMap &,
                                       const CUtensorMap &, int, int *, cudaStream_t,
                                       const SideStream *);
template cudaError_t launch_tma<double>(const FusedArgs<double> &, const CUtensorMap &,
                                        const CUtensorMap &, int, int *, cudaStream_t,
                                        const SideStream *);

}  // namespace yf
