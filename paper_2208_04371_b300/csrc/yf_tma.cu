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
// outside the grid arrive as zeros (TMA out-of-bounds fill).  Every thread waits on the
// stage's mbarrier itself, and every wait is bounded: a thread whose wait expires finishes the
// plane, then the block sets bit 1 of the status word and returns together at the plane's end
// barrier.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

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
    // CPML profiles of the block: x [6][BX], y [6][WY], z [6][ZMAX] (planes kb-1 .. ke)
    static constexpr int ZMAX = kMaxKseg + 2;
    static constexpr int PR_OFF = BAR_OFF + 64;
    static constexpr int PR_BYTES = (6 * (BX + WY + ZMAX) * (int)sizeof(T) + 15) / 16 * 16;
    static constexpr int BYTES = PR_OFF + PR_BYTES;
    static constexpr uint32_t TX_BYTES = 2 * WIN_BYTES + CLS_BYTES;
};

template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// CPML term from a staged profile: pr holds b, a, 1/kappa at integer nodes (rows 0..2) and at
// half nodes (rows 3..5), `stride` entries per row.  psi_new = b psi + a d (stored at w when
// given); returns d / kappa + psi_new.
template <typename T>
__device__ __forceinline__ T cpt(T d, T psi, T *w, const T *pr, int stride, int which, int idx)
{
    const T v = pr[which * stride + idx] * psi + pr[(which + 1) * stride + idx] * d;
    if (w) *w = v;
    return d * pr[(which + 2) * stride + idx] + v;
}

// Block: TX x TYT threads; thread (tx, ty) owns node column i = i0 + tx and the CY rows
// j = j0 + ty*CY + r (r < CY) of a TX x (TYT*CY) tile.  Rows of one thread are contiguous, so
// the y neighbours of its E and H values come from registers, E^n read for the H update is
// reused by the E update, and the loop overhead of a plane is paid once per CY nodes.
// HP (absorbing slabs present): the block's CPML profiles sit in shared memory and each
// thread fetches the auxiliaries of plane p+1 while it computes plane p.
template <typename T, int TX, int TYT, int CY, int PM>
__device__ __forceinline__ void tma_tile(const FusedArgs<T> &P, const CUtensorMap *tmF,
                                         const CUtensorMap *tmC, int *status, unsigned char *sm,
                                         int i0, int j0, int kb, int ke)
{
    constexpr int TY = TYT * CY;
    // PM: CPML code compiled in for the x (1), y (2) and z (4) slabs
    constexpr bool HPX = (PM & 1) != 0, HPY = (PM & 2) != 0, HPZ = (PM & 4) != 0;
    constexpr bool HP = PM != 0;
    using Lay = TmaLayout<T, TX, TY>;
    using P2 = typename Pair<T>::type;
    constexpr int XO = Lay::XO, BX = Lay::BX, WN = Lay::WN, WY = Lay::WY, NT = TX * TYT;
    constexpr int ZMAX = Lay::ZMAX;
    T *sHn = reinterpret_cast<T *>(sm + Lay::SH_OFF);
    P2 *sC = reinterpret_cast<P2 *>(sm + Lay::CT_OFF);
    T *PX = reinterpret_cast<T *>(sm + Lay::PR_OFF);   // [6][BX]
    T *PY = PX + 6 * BX;                                  // [6][WY]
    T *PZ = PY + 6 * WY;                                  // [6][ZMAX]
    const uint32_t bar0 = smem_u32(sm + Lay::BAR_OFF);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i = i0 + tx, jb = j0 + ty * CY;
    const long plane = P.plane, npts = P.npts;
    // arguments the plane loop uses, held in registers (the shared copy would be re-read after
    // every barrier)
    const T rdx = P.rdx, rdy = P.rdy, rdz = P.rdz, db = P.db;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    T *const Bo = P.B;
    const int px = P.px, NX1 = nx + 1, NY1 = ny + 1;
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
    if (HPX) {
        for (int q = tid; q < 6 * BX; q += NT) {
            const int k = q / BX, gi = i0 - XO + q % BX;
            PX[q] = (P.prof[0] && gi >= 0 && gi <= nx) ? P.prof[0][k * NX1 + gi] : (T)0;
        }
    }
    if (HPY) {
        for (int q = tid; q < 6 * WY; q += NT) {
            const int k = q / WY, gj = j0 - 1 + q % WY;
            PY[q] = (P.prof[1] && gj >= 0 && gj <= ny) ? P.prof[1][k * NY1 + gj] : (T)0;
        }
    }
    if (HPZ) {
        for (int q = tid; q < 6 * ZMAX; q += NT) {
            const int k = q / ZMAX, gp = kb - 1 + q % ZMAX;
            PZ[q] = (P.prof[2] && gp >= 0 && gp <= nz) ? P.prof[2][k * (nz + 1) + gp] : (T)0;
        }
    }
    __syncthreads();

    // plane q lives in stage (q - kb + 1) mod 3; thread 0 tracks the parity of each stage's
    // next completion in `phase` (bit s)
    auto issue = [&](int q, int s) {   // thread 0 only
        unsigned char *st = sm + s * Lay::STAGE;
        const uint32_t bar = bar0 + 8 * s;
        mbar_expect_tx(bar, Lay::TX_BYTES);
        tma_load_4d(smem_u32(st), tmF, i0 - XO, j0 - 1, q, 0, bar);
        tma_load_4d(smem_u32(st + Lay::WIN_PAD), tmF, i0 - XO, j0 - 1, q, 3, bar);
        tma_load_4d(smem_u32(st + 2 * Lay::WIN_PAD), tmC, i0, j0, q, 0, bar);
    };
    uint32_t phase = 0;
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int q = kb - 1, s = 0; q <= kb + 1 && q <= ke + 1; ++q, ++s) issue(q, s);
    }
    // first plane: one thread polls the stage barrier, the others sleep in the block barrier
    // (every thread keeps the phase bits)
    auto wait_stage = [&](int s) -> bool {
        bool ok = true;
        if (tid == 0) ok = mbar_wait(bar0 + 8 * s, (phase >> s) & 1u);
        phase ^= 1u << s;
        return __syncthreads_and(ok);
    };
    if (!wait_stage(0)) {
        if (tid == 0) atomicOr(status, 2);
        return;
    }

    // per-thread constants
    const bool col_live = i <= nx;
    const int sx = HPX ? slab_i(i, nx, n, P.lo[0], P.hi[0]) : -1;
    const int lx = tx + XO;            // staged x-profile index of the own column
    int sy[CY];
    bool rlive[CY];
#pragma unroll
    for (int r = 0; r < CY; ++r) {
        sy[r] = HPY ? slab_i(jb + r, ny, n, P.lo[1], P.hi[1]) : -1;
        rlive[r] = col_live && jb + r <= ny;
    }
    const int w0 = (ty * CY + 1) * BX + (tx + XO);   // window index of row r: w0 + r * BX

    // halo value owned by this thread (threads 0 .. 2TX+2TY-1): the row j0-1 needs H_x and
    // H_z for i0 <= i < i0+TX, the column i0-1 needs H_y and H_z for j0 <= j < j0+TY.
    // h_comp: 0 H_x, 1 H_y, 2 H_z, -1 none; h_live false stores a zero (outside the grid)
    constexpr int NHALO = 2 * TX + 2 * TY;
    static_assert(NHALO <= NT, "one halo value per thread");
    int h_comp = -1, h_w = 0, h_i = 0, h_j = 0, h_sx = -1, h_sy = -1, h_lx = 0, h_ly = 0;
    bool h_live = false;
    if (tid < NHALO) {
        if (tid < 2 * TX) {
            const int e = tid < TX ? tid : tid - TX;
            h_comp = tid < TX ? 0 : 2;
            h_w = e + XO;
            h_i = i0 + e;
            h_j = j0 - 1;
            h_lx = e + XO;
            h_ly = 0;
            h_live = j0 > 0 && h_i <= nx;
        } else {
            const int e = tid - 2 * TX;
            const int r = e < TY ? e : e - TY;
            h_comp = e < TY ? 1 : 2;
            h_w = (r + 1) * BX + (XO - 1);
            h_i = i0 - 1;
            h_j = j0 + r;
            h_lx = XO - 1;
            h_ly = r + 1;
            h_live = i0 > 0 && h_j <= ny;
        }
        if (HPX && h_live) h_sx = slab_i(h_i, nx, n, P.lo[0], P.hi[0]);
        if (HPY && h_live) h_sy = slab_i(h_j, ny, n, P.lo[1], P.hi[1]);
    }

    // CPML auxiliaries of plane q for the own rows (pv) and the halo value (hv):
    //   pv[r][0..3]  y slab: H_x, H_z, E_x, E_z    offset (q L + sy) px + i
    //   pv[r][4..7]  z slab: H_x, H_y, E_x, E_y    offset (sz NY1 + j) px + i
    //   pv[r][8..11] x slab: H_y, H_z, E_y, E_z    offset (q NY1 + j) L + sx
    // fetched one plane ahead; the H values come from the read copy, the E values are the
    // thread's own (updated in place by this thread only)
    T pv[CY][12];
    T hv[2] = {0, 0};
    auto fetch = [&](int q) {
        if (!HP || q < 0 || q > nz) return;
        const int szq = HPZ ? slab_i(q, nz, n, P.lo[2], P.hi[2]) : -1;
#pragma unroll
        for (int r = 0; r < CY; ++r) {
            const int j = jb + r;
            if (!rlive[r]) continue;
            if (HPY && sy[r] >= 0) {
                const int o = (q * L + sy[r]) * px + i;
                pv[r][0] = P.psiHr[1][0][o]; pv[r][1] = P.psiHr[1][1][o];
                pv[r][2] = P.psiE[1][0][o];  pv[r][3] = P.psiE[1][1][o];
            }
            if (HPZ && szq >= 0) {
                const int o = (szq * NY1 + j) * px + i;
                pv[r][4] = P.psiHr[2][0][o]; pv[r][5] = P.psiHr[2][1][o];
                pv[r][6] = P.psiE[2][0][o];  pv[r][7] = P.psiE[2][1][o];
            }
            if (HPX && sx >= 0) {
                const int o = (q * NY1 + j) * L + sx;
                pv[r][8] = P.psiHr[0][0][o];  pv[r][9] = P.psiHr[0][1][o];
                pv[r][10] = P.psiE[0][0][o];  pv[r][11] = P.psiE[0][1][o];
            }
        }
        if (h_live && q >= kb) {
            // the two terms of the halo value: (first derivative, second derivative)
            const int ys = h_sy >= 0 ? (q * L + h_sy) * px + h_i : 0;
            const int zs = szq >= 0 ? (szq * NY1 + h_j) * px + h_i : 0;
            const int xs = h_sx >= 0 ? (q * NY1 + h_j) * L + h_sx : 0;
            if (h_comp == 0) {          // H_x: y then z
                if (h_sy >= 0) hv[0] = P.psiHr[1][0][ys];
                if (szq >= 0) hv[1] = P.psiHr[2][0][zs];
            } else if (h_comp == 1) {   // H_y: z then x
                if (szq >= 0) hv[0] = P.psiHr[2][1][zs];
                if (h_sx >= 0) hv[1] = P.psiHr[0][0][xs];
            } else {                    // H_z: x then y
                if (h_sx >= 0) hv[0] = P.psiHr[0][1][xs];
                if (h_sy >= 0) hv[1] = P.psiHr[1][1][ys];
            }
        }
    };
#pragma unroll
    for (int r = 0; r < CY; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) pv[r][k] = 0;
    fetch(kb - 1);

    T hx_prev[CY], hy_prev[CY];
#pragma unroll
    for (int r = 0; r < CY; ++r) hx_prev[r] = hy_prev[r] = 0;
    int sp = 0, sn = 1;   // stages of planes p and p + 1
    bool gave_up = false;
    for (int p = kb - 1; p <= ke; ++p) {
        // plane p + 1 must have landed (its E is the upper neighbour of plane p's H).  Every
        // thread waits on the stage barrier itself: the end-of-plane barrier below already
        // orders the last plane's reads of sHn before this plane's writes.  A thread whose
        // wait gives up carries on (its results are discarded) and the block leaves together
        // at that barrier.
        gave_up |= !mbar_wait(bar0 + 8 * sn, (phase >> sn) & 1u);
        phase ^= 1u << sn;
        const unsigned char *stp = sm + sp * Lay::STAGE;
        const unsigned char *stn = sm + sn * Lay::STAGE;
        const T *ex0 = reinterpret_cast<const T *>(stp), *ey0 = ex0 + WN, *ez0 = ey0 + WN;
        const T *hox = reinterpret_cast<const T *>(stp + Lay::WIN_PAD), *hoy = hox + WN, *hoz = hoy + WN;
        const uint8_t *cl = stp + 2 * Lay::WIN_PAD;
        const T *ex1 = reinterpret_cast<const T *>(stn), *ey1 = ex1 + WN;
        const bool pin = p >= 0;
        const int sz = (HPZ && pin) ? slab_i(p, nz, n, P.lo[2], P.hi[2]) : -1;
        const int lz = p - kb + 1;   // staged z-profile index of plane p

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
            if (pin && p < nz) {
#pragma unroll
                for (int r = 0; r < CY; ++r) {
                    const int w = w0 + r * BX, ly = ty * CY + r + 1;
                    T d1 = (ezv[r + 1] - ezv[r]) * rdy, d2 = (ey1v[r] - eyv[r]) * rdz;
                    if (HPY && sy[r] >= 0) d1 = cpt(d1, pv[r][0], (T *)nullptr, PY, WY, 3, ly);
                    if (HPZ && sz >= 0) d2 = cpt(d2, pv[r][4], (T *)nullptr, PZ, ZMAX, 3, lz);
                    hx_prev[r] = hox[w] - db * (d1 - d2);
                    d1 = (ex1v[r] - exv[r]) * rdz;
                    d2 = (ezx[r] - ezv[r]) * rdx;
                    if (HPZ && sz >= 0) d1 = cpt(d1, pv[r][5], (T *)nullptr, PZ, ZMAX, 3, lz);
                    if (HPX && sx >= 0) d2 = cpt(d2, pv[r][8], (T *)nullptr, PX, BX, 3, lx);
                    hy_prev[r] = hoy[w] - db * (d1 - d2);
                }
            }
        } else {
            const long qb = (long)p * plane + (long)jb * px + i;
            T hx[CY], hy[CY], hz[CY];
#pragma unroll
            for (int r = 0; r < CY; ++r) {
                const int w = w0 + r * BX, j = jb + r, ly = ty * CY + r + 1;
                const bool vx = rlive[r] && j < ny && p < nz;
                const bool vy = rlive[r] && i < nx && p < nz;
                const bool vz = rlive[r] && i < nx && j < ny;
                // H_x(i, j+1/2, p+1/2) -= dt/mu0 (dEz/dy - dEy/dz)
                T d1 = (ezv[r + 1] - ezv[r]) * rdy, d2 = (ey1v[r] - eyv[r]) * rdz;
                if (HPY && sy[r] >= 0)
                    d1 = cpt(d1, pv[r][0], vx ? P.psiHw[1][0] + (p * L + sy[r]) * px + i : (T *)nullptr, PY, WY, 3, ly);
                if (HPZ && sz >= 0)
                    d2 = cpt(d2, pv[r][4], vx ? P.psiHw[2][0] + (sz * NY1 + j) * px + i : (T *)nullptr, PZ, ZMAX, 3, lz);
                hx[r] = hox[w] - db * (d1 - d2);
                // H_y(i+1/2, j, p+1/2) -= dt/mu0 (dEx/dz - dEz/dx)
                d1 = (ex1v[r] - exv[r]) * rdz;
                d2 = (ezx[r] - ezv[r]) * rdx;
                if (HPZ && sz >= 0)
                    d1 = cpt(d1, pv[r][5], vy ? P.psiHw[2][1] + (sz * NY1 + j) * px + i : (T *)nullptr, PZ, ZMAX, 3, lz);
                if (HPX && sx >= 0)
                    d2 = cpt(d2, pv[r][8], vy ? P.psiHw[0][0] + (p * NY1 + j) * L + sx : (T *)nullptr, PX, BX, 3, lx);
                hy[r] = hoy[w] - db * (d1 - d2);
                // H_z(i+1/2, j+1/2, p) -= dt/mu0 (dEy/dx - dEx/dy)
                d1 = (eyx[r] - eyv[r]) * rdx;
                d2 = (exv[r + 1] - exv[r]) * rdy;
                if (HPX && sx >= 0)
                    d1 = cpt(d1, pv[r][9], vz ? P.psiHw[0][1] + (p * NY1 + j) * L + sx : (T *)nullptr, PX, BX, 3, lx);
                if (HPY && sy[r] >= 0)
                    d2 = cpt(d2, pv[r][1], vz ? P.psiHw[1][1] + (p * L + sy[r]) * px + i : (T *)nullptr, PY, WY, 3, ly);
                hz[r] = hoz[w] - db * (d1 - d2);
                sHn[w] = hx[r];
                sHn[WN + w] = hy[r];
                sHn[2 * WN + w] = hz[r];
                const long q = qb + (long)r * px;
                if (vx) Bo[3 * npts + q] = hx[r];
                if (vy) Bo[4 * npts + q] = hy[r];
                if (vz) Bo[5 * npts + q] = hz[r];
            }
            if (h_comp >= 0) {   // one halo H value per thread of the first warps
                T v = 0;
                if (h_live) {
                    const int w = h_w;
                    if (h_comp == 0) {
                        T d1 = (ez0[w + BX] - ez0[w]) * rdy, d2 = (ey1[w] - ey0[w]) * rdz;
                        if (HPY && h_sy >= 0) d1 = cpt(d1, hv[0], (T *)nullptr, PY, WY, 3, h_ly);
                        if (HPZ && sz >= 0) d2 = cpt(d2, hv[1], (T *)nullptr, PZ, ZMAX, 3, lz);
                        v = hox[w] - db * (d1 - d2);
                    } else if (h_comp == 1) {
                        T d1 = (ex1[w] - ex0[w]) * rdz, d2 = (ez0[w + 1] - ez0[w]) * rdx;
                        if (HPZ && sz >= 0) d1 = cpt(d1, hv[0], (T *)nullptr, PZ, ZMAX, 3, lz);
                        if (HPX && h_sx >= 0) d2 = cpt(d2, hv[1], (T *)nullptr, PX, BX, 3, h_lx);
                        v = hoy[w] - db * (d1 - d2);
                    } else {
                        T d1 = (ey0[w + 1] - ey0[w]) * rdx, d2 = (ex0[w + BX] - ex0[w]) * rdy;
                        if (HPX && h_sx >= 0) d1 = cpt(d1, hv[0], (T *)nullptr, PX, BX, 3, h_lx);
                        if (HPY && h_sy >= 0) d2 = cpt(d2, hv[1], (T *)nullptr, PY, WY, 3, h_ly);
                        v = hoz[w] - db * (d1 - d2);
                    }
                }
                sHn[h_comp * WN + h_w] = v;
            }
            __syncthreads();

            const T *shx = sHn, *shy = sHn + WN, *shz = sHn + 2 * WN;
            T hz_up = shz[w0 - BX], hx_up = shx[w0 - BX];
#pragma unroll
            for (int r = 0; r < CY; ++r) {
                const int w = w0 + r * BX, j = jb + r, ly = ty * CY + r + 1;
                const int crow = (ty * CY + r) * TX + tx;
                T exn = 0, eyn = 0, ezn = 0;
                int c = cl[crow];
                if (c) {   // E_x(i+1/2, j, p) = Ca E_x + Cb (dHz/dy - dHy/dz)
                    T d1 = (hz[r] - hz_up) * rdy, d2 = (hy[r] - hy_prev[r]) * rdz;
                    if (HPY && sy[r] >= 0) d1 = cpt(d1, pv[r][2], P.psiE[1][0] + (p * L + sy[r]) * px + i, PY, WY, 0, ly);
                    if (HPZ && sz >= 0) d2 = cpt(d2, pv[r][6], P.psiE[2][0] + (sz * NY1 + j) * px + i, PZ, ZMAX, 0, lz);
                    const P2 k = sC[c];
                    exn = k.x * exv[r] + k.y * (d1 - d2);
                }
                c = cl[TX * TY + crow];
                if (c) {   // E_y(i, j+1/2, p) = Ca E_y + Cb (dHx/dz - dHz/dx)
                    T d1 = (hx[r] - hx_prev[r]) * rdz, d2 = (hz[r] - shz[w - 1]) * rdx;
                    if (HPZ && sz >= 0) d1 = cpt(d1, pv[r][7], P.psiE[2][1] + (sz * NY1 + j) * px + i, PZ, ZMAX, 0, lz);
                    if (HPX && sx >= 0) d2 = cpt(d2, pv[r][10], P.psiE[0][0] + (p * NY1 + j) * L + sx, PX, BX, 0, lx);
                    const P2 k = sC[c];
                    eyn = k.x * eyv[r] + k.y * (d1 - d2);
                }
                c = cl[2 * TX * TY + crow];
                if (c) {   // E_z(i, j, p+1/2) = Ca E_z + Cb (dHy/dx - dHx/dy)
                    T d1 = (hy[r] - shy[w - 1]) * rdx, d2 = (hx[r] - hx_up) * rdy;
                    if (HPX && sx >= 0) d1 = cpt(d1, pv[r][11], P.psiE[0][1] + (p * NY1 + j) * L + sx, PX, BX, 0, lx);
                    if (HPY && sy[r] >= 0) d2 = cpt(d2, pv[r][3], P.psiE[1][1] + (p * L + sy[r]) * px + i, PY, WY, 0, ly);
                    const P2 k = sC[c];
                    ezn = k.x * ezv[r] + k.y * (d1 - d2);
                }
                if (rlive[r]) {
                    const long q = qb + (long)r * px;
                    Bo[q] = exn;
                    Bo[npts + q] = eyn;
                    Bo[2 * npts + q] = ezn;
                }
                hz_up = hz[r];
                hx_up = hx[r];
                hx_prev[r] = hx[r];
                hy_prev[r] = hy[r];
            }
        }
        // auxiliaries of the next plane, in flight during the barrier and the next wait
        fetch(p + 1);
        // every thread is done with stage sp: refill it with plane p + 3
        if (__syncthreads_or(gave_up)) {
            if (tid == 0) atomicOr(status, 2);
            return;
        }
        if (tid == 0 && p + 3 <= ke + 1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(p + 3, sp);
        }
        sp = sn;
        sn = sn == Lay::NST - 1 ? 0 : sn + 1;
    }
}

// Block b takes work item b (instance, tile origin, z-segment); the instance's arguments for
// the current buffer parity are copied to shared memory behind the TMA layout.  FP32 kinds
// with one row per thread are held to five resident blocks per SM (the shared-memory limit;
// 48 registers), the all-CPML kind to four (64); FP64 and two-row tiles keep the compiler's
// choice (a cap would spill).
template <typename T, int TX, int TYT, int CY, int PM>
__global__ void __launch_bounds__(TX *TYT, (sizeof(T) == 4 && CY == 1) ? ((PM == 7) ? 4 : 5) : 1)
    k_yee_tma_batch(const BatchItem *items, const FusedArgs<T> *args, const CUtensorMap *maps,
                    int parity, int stride, int *status)
{
    extern __shared__ __align__(128) unsigned char sm[];
    using Lay = TmaLayout<T, TX, TYT * CY>;
    static_assert(Lay::BYTES % 16 == 0, "argument copy alignment");
    const BatchItem it = items[blockIdx.x];
    FusedArgs<T> *sP = reinterpret_cast<FusedArgs<T> *>(sm + Lay::BYTES);
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int *src = reinterpret_cast<const int *>(args + stride * it.inst + parity);
    int *dst = reinterpret_cast<int *>(sP);
    for (int q = tid; q < (int)(sizeof(FusedArgs<T>) / 4); q += TX * TYT) dst[q] = src[q];
    __syncthreads();
    const CUtensorMap *m = maps + 2 * (stride * it.inst + parity);
    tma_tile<T, TX, TYT, CY, PM>(*sP, m, m + 1, status, sm, it.i0, it.j0, it.kb, it.ke);
}

template <typename T, int TX, int TYT, int CY, int PM>
int batch_bytes()
{
    return TmaLayout<T, TX, TYT * CY>::BYTES + (int)sizeof(FusedArgs<T>);
}

template <typename T, int TX, int TYT, int CY, int PM>
cudaError_t prep_one()
{
    return cudaFuncSetAttribute(k_yee_tma_batch<T, TX, TYT, CY, PM>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                batch_bytes<T, TX, TYT, CY, PM>());
}

template <typename T, int TX, int TYT, int CY>
cudaError_t prep_kinds()
{
    cudaError_t e;
    if ((e = prep_one<T, TX, TYT, CY, 0>()) != cudaSuccess) return e;
    if ((e = prep_one<T, TX, TYT, CY, 1>()) != cudaSuccess) return e;
    if ((e = prep_one<T, TX, TYT, CY, 2>()) != cudaSuccess) return e;
    if ((e = prep_one<T, TX, TYT, CY, 4>()) != cudaSuccess) return e;
    return prep_one<T, TX, TYT, CY, 7>();
}

template <typename T, int TX, int TYT, int CY, int PM>
cudaError_t launch_kind(const TmaPlan &pl, int kind, int parity, int *status, cudaStream_t s)
{
    const int cnt = pl.count[kind];
    if (cnt <= 0) return cudaSuccess;
    k_yee_tma_batch<T, TX, TYT, CY, PM><<<cnt, dim3(TX, TYT), batch_bytes<T, TX, TYT, CY, PM>(), s>>>(
        pl.items + pl.offset[kind], (const FusedArgs<T> *)pl.args, pl.maps, parity, pl.stride > 0 ? pl.stride : 2,
        status);
    return cudaGetLastError();
}

template <typename T, int TX, int TYT, int CY>
cudaError_t launch_plan_t(const TmaPlan &pl, int parity, int *status, cudaStream_t s,
                          const SideStream *side)
{
    // kind 0 (no CPML) on the main stream; each CPML kind on its own side stream, so the four
    // small frame launches overlap one another and the interior
    cudaError_t e;
    const bool frame = pl.count[1] + pl.count[2] + pl.count[3] + pl.count[4] > 0;
    const bool fork = frame && side && side->ready;
    if (fork && (e = cudaEventRecord(side->fork, s)) != cudaSuccess) return e;
    const int kinds[kSideStreams] = {4, 1, 2, 3};
    bool joined[kSideStreams] = {false, false, false, false};
    for (int q = 0; q < kSideStreams; ++q) {
        const int kind = kinds[q];
        if (pl.count[kind] <= 0) continue;
        cudaStream_t fs = s;
        if (fork) {
            fs = side->stream[q];
            if ((e = cudaStreamWaitEvent(fs, side->fork, 0)) != cudaSuccess) return e;
        }
        switch (kind) {
        case 4: e = launch_kind<T, TX, TYT, CY, 7>(pl, 4, parity, status, fs); break;
        case 1: e = launch_kind<T, TX, TYT, CY, 1>(pl, 1, parity, status, fs); break;
        case 2: e = launch_kind<T, TX, TYT, CY, 2>(pl, 2, parity, status, fs); break;
        default: e = launch_kind<T, TX, TYT, CY, 4>(pl, 3, parity, status, fs); break;
        }
        if (e != cudaSuccess) return e;
        if (fork) {
            if ((e = cudaEventRecord(side->join[q], fs)) != cudaSuccess) return e;
            joined[q] = true;
        }
    }
    if ((e = launch_kind<T, TX, TYT, CY, 0>(pl, 0, parity, status, s)) != cudaSuccess) return e;
    for (int q = 0; q < kSideStreams; ++q)
        if (joined[q] && (e = cudaStreamWaitEvent(s, side->join[q], 0)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace

cudaError_t side_create(SideStream *s)
{
    if (s->ready) return cudaSuccess;
    cudaError_t e;
    for (int q = 0; q < kSideStreams; ++q) {
        if ((e = cudaStreamCreateWithFlags(&s->stream[q], cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&s->join[q], cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    if ((e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    s->ready = true;
    return cudaSuccess;
}

void side_destroy(SideStream *s)
{
    if (!s->ready) return;
    for (int q = 0; q < kSideStreams; ++q) {
        cudaStreamSynchronize(s->stream[q]);
        cudaEventDestroy(s->join[q]);
        cudaStreamDestroy(s->stream[q]);
    }
    cudaEventDestroy(s->fork);
    s->ready = false;
}

template <typename T>
int tma_box_x(int tile_x) { return tile_x + 2 * (16 / (int)sizeof(T)); }

// shared-memory opt-in of every instantiation; call outside stream capture
cudaError_t tma_prepare()
{
    cudaError_t e;
    if ((e = prep_kinds<float, 32, 4, 1>()) != cudaSuccess) return e;
    if ((e = prep_kinds<float, 32, 8, 1>()) != cudaSuccess) return e;
    if ((e = prep_kinds<float, 32, 8, 2>()) != cudaSuccess) return e;
    if ((e = prep_kinds<double, 32, 4, 1>()) != cudaSuccess) return e;
    if ((e = prep_kinds<double, 32, 8, 1>()) != cudaSuccess) return e;
    return prep_kinds<double, 32, 8, 2>();
}

// tile_y = rows per block: 4 -> 4 threads x 1 row, 8 -> 8 x 1, 16 -> 8 x 2
template <typename T>
cudaError_t launch_tma_plan(const TmaPlan &pl, int tile_y, int parity, int *status, cudaStream_t s,
                            const SideStream *side)
{
    switch (tile_y) {
    case 4: return launch_plan_t<T, 32, 4, 1>(pl, parity, status, s, side);
    case 16: return launch_plan_t<T, 32, 8, 2>(pl, parity, status, s, side);
    default: return launch_plan_t<T, 32, 8, 1>(pl, parity, status, s, side);
    }
}

// Work items of one grid for tile height tile_y.  The interior box (tiles whose nodes and halo
// nodes avoid the x and y slabs, planes from the warm-up plane on outside the z slabs) is kind
// 0; tiles outside it in x only -> kind 1 (x CPML), in y only -> kind 2, in z only -> kind 3
// (z CPML), anything else -> kind 4 (all CPML).  z segments never straddle the z-slab limits.
void tma_items(int inst, int nx, int ny, int nz, int kseg, int tile_y, int n, const int lo[3],
               const int hi[3], std::vector<BatchItem> items[5], int mixed_seg)
{
    // Tiles cover node columns 0 .. nx-1 and rows 0 .. ny-1.  The last node column i = nx
    // (and row j = ny) joins a tile only when nx (ny) is not a multiple of the tile: on that
    // PEC-backed face the tangential E are zero and the only H there (H_x at i = nx, H_y at
    // j = ny) keeps its value, so a tile holding nothing else is skipped (the two field
    // buffers hold equal values there: the write and checkpoint-load calls fill both).
    const int TX = 32, TY = tile_y;
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY;
    const bool hp = n > 0 && (lo[0] || hi[0] || lo[1] || hi[1] || lo[2] || hi[2]);
    auto lo_tile = [](int on, int n_, int tile) { return on ? (n_ + 1 + tile - 1) / tile : 0; };
    auto hi_tile = [](int on, int N, int n_, int tile, int count) {
        if (!on) return count;
        const int lim = N - n_ - tile;   // largest origin with origin + tile - 1 < N - n
        return lim < 0 ? 0 : lim / tile + 1;
    };
    int txa = 0, txb = ntx, tya = 0, tyb = nty, za = 0, zb = nz;
    if (hp) {
        txa = lo_tile(lo[0] && n > 0, n, TX); txb = std::min(ntx, hi_tile(hi[0] && n > 0, nx, n, TX, ntx));
        tya = lo_tile(lo[1] && n > 0, n, TY); tyb = std::min(nty, hi_tile(hi[1] && n > 0, ny, n, TY, nty));
        za = lo[2] ? n + 1 : 0;
        zb = hi[2] ? nz - n - 1 : nz;
    }
    // z segments (the same for every tile of the grid), outermost, so that blocks launched
    // together are x/y neighbours on the same planes and share halo rows through L2
    std::vector<std::pair<int, int>> segs;
    for (int k = 0; k <= nz;) {
        const bool inz = k >= za && k <= zb;
        const int stop = inz ? zb : (k < za ? za - 1 : nz);
        const int kend = std::min(stop, k + kseg - 1);
        segs.push_back({k, kend});
        k = kend + 1;
    }
    for (const auto &sg : segs) {
        const bool inz = sg.first >= za && sg.first <= zb;
        for (int ty = 0; ty < nty; ++ty)
            for (int tx = 0; tx < ntx; ++tx) {
                const bool inx = tx >= txa && tx < txb, iny = ty >= tya && ty < tyb;
                int kind;
                if (!hp) kind = 0;
                else if (inz) kind = inx ? (iny ? 0 : 2) : (iny ? 1 : 4);
                else kind = (inx && iny) ? 3 : 4;
                if (kind == 4 && mixed_seg > 0) {
                    // where the all-CPML kind is small (one large grid), shorter segments give
                    // it more blocks and a shorter longest block
                    for (int k0 = sg.first; k0 <= sg.second; k0 += mixed_seg)
                        items[kind].push_back(BatchItem{inst, tx * TX, ty * TY, k0, std::min(sg.second, k0 + mixed_seg - 1)});
                    continue;
                }
                items[kind].push_back(BatchItem{inst, tx * TX, ty * TY, sg.first, sg.second});
            }
    }
}

template int tma_box_x<float>(int);
template int tma_box_x<double>(int);
template cudaError_t launch_tma_plan<float>(const TmaPlan &, int, int, int *, cudaStream_t,
                                            const SideStream *);
template cudaError_t launch_tma_plan<double>(const TmaPlan &, int, int, int *, cudaStream_t,
                                             const SideStream *);

}  // namespace yf
