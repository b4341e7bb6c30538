// Two-step (temporally blocked) Yee update of the inner box, FP32 (variant 4).
//
// The inner box is a set of whole 32 x 8 tiles and a z range that keep at least three nodes
// from every CPML slab and domain wall and four from the source and port planes, so only the
// plain Yee update (materials through the class table) happens in and around it.  One block
// takes one tile over a z segment [kb, ke] and advances it from step n (buffer A) to step
// n + 2 (buffer C) in one pass over HBM:
//   S1  H^{n+1/2}  on the tile grown by 2 nodes on the low sides, 1 on the high sides
//   S2  E^{n+1}    on the tile grown by 1 node on every side
//   S3  H^{n+3/2}  on the tile grown by 1 node on the low sides
//   S4  E^{n+2}    on the tile, written to C together with H^{n+3/2}
// The grown rings recompute, from the same step-n data, what neighbouring blocks (or the
// single-step frame) own.  Threads work on x-pairs of nodes, so some regions reach one node
// further; those extra nodes feed nothing.
//
// z is marched with the stages skewed so that each plane iteration q has two phases separated
// by one block barrier: {S1 on plane q-1, S3 on plane q-3}, then {S2 on plane q-1, S4 on
// plane q-3}; every input of a phase comes from an earlier phase.  Step-n planes arrive by TMA
// two planes ahead (the last warp, idle in the second phase, issues each refill there): E and
// H windows of 40 x 12 nodes (x from i0-4, y from j0-2) in four stages, the class tiles
// (80 x 10 bytes) in six slots (S4 reads the classes of plane q-3).  H^{n+1/2} and E^{n+1} are
// kept for three planes, H^{n+3/2} for two, in rings over the same nodes with rows of 44
// floats, so that the strip tasks of eight rows fall in distinct banks.
//
// The single-step frame advances the rest of the grid n -> n+1 (A -> B) and n+1 -> n+2
// (B -> C).  Its second step reads the box's outermost node layer at n + 1 from B (a window
// reaches one node into the box), so this kernel also writes E^{n+1} and H^{n+1/2} of that
// layer into B.  Every mbarrier wait is bounded; a wait that gives up sets bit 1 of the status
// word and the block returns.  The host side (box, work items, arguments, the pair of steps)
// is in yf_tb_plan.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "yf_internal.h"

namespace yf {
namespace {

constexpr int TBX = kTbTileX, TBY = kTbTileY;         // output tile
constexpr int NWARP = 12, TBN = 32 * NWARP;          // block
constexpr int WXN = kTbWinX, WYN = kTbWinY, WN = WXN * WYN;   // windows: x from i0-4, y from j0-2
// the rings the threads write (H^{n+1/2}, E^{n+1}, H^{n+3/2}) cover the same nodes with rows of
// 44 floats: a 12-bank shift per row spreads the strips of eight rows over all 32 banks
constexpr int WXR = 44, WR = WXR * WYN;
constexpr int CXN = kTbClsX, CYN = kTbClsY, CN = CXN * CYN;   // class tile: x from i0-16, y from j0-1
constexpr int CSLOT = (3 * CN + 127) / 128 * 128;    // one class slot (bytes)
constexpr int FST = 4, CSL = 6;                      // field stages, class slots
constexpr int PL = 3 * WN * 4;                       // one stage plane of three components (bytes)
constexpr int PR = 3 * WR * 4;                       // one ring plane of three components (bytes)
constexpr int C_OFF = FST * 2 * PL;                  // stage s: E at s * 2PL, H at s * 2PL + PL
constexpr int HA_OFF = C_OFF + CSL * CSLOT;          // H^{n+1/2} [3][3][WR]
constexpr int EA_OFF = HA_OFF + 3 * PR;              // E^{n+1}   [3][3][WR]
constexpr int HB_OFF = EA_OFF + 3 * PR;              // H^{n+3/2} [2][3][WR]
constexpr int CT_OFF = HB_OFF + 2 * PR;              // (Ca, Cb) per class
constexpr int BAR_OFF = CT_OFF + 2 * kMaxClasses * 4;
constexpr int TB_BYTES = BAR_OFF + 8 * FST;
constexpr uint32_t TX_BYTES = 2 * PL + 3 * CN;
static_assert(PL % 128 == 0 && C_OFF % 128 == 0 && CSLOT % 128 == 0, "TMA destinations 128-byte aligned");
static_assert(PR % 16 == 0 && HA_OFF % 16 == 0, "ring planes 16-byte aligned");
static_assert(2 * (TB_BYTES + 1024) <= 228 * 1024, "two blocks per SM");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 26); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int c,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(c), "r"(bar)
        : "memory");
}

// Each thread updates one pair of x-adjacent nodes (i, i+1), i - i0 even, per phase.  A
// half-warp takes the first 16 pairs of one row (128 contiguous bytes, no bank conflicts);
// the one or two pairs left at the right end of each row form short strips:
//   phase 1: threads   0..175 S1 rows j0-2..j0+8, pairs 0..15 from i0-2;  176..197 pairs 16, 17
//            threads 224..367 S3 rows j0-1..j0+7, pairs 0..15 from i0-2;  368..376 pair 16
//   phase 2: threads   0..159 S2 rows j0-1..j0+8, pairs 0..15 from i0-2;  160..179 pairs 16, 17
//            threads 192..319 S4 rows j0..j0+7,   pairs 0..15 from i0
// so every warp runs one stage.  Pairs reach one node past the needed ranges on the left of
// S2 and S3 and on the right of S1 and S2; those extra nodes read neighbours nobody computed
// and feed nothing.  The pair's values move as float2 (64-bit shared loads, one 32-bit load
// for the neighbour shifted by one node in x) through Blackwell's paired FP32 arithmetic.
// w, v, c: window, ring and class-tile index of the pair's first node; g: its offset j px + i in a
// field plane; own: the pair is in the block's tile; lay: a node of it lies on the box's
// outer layer in x or y.
struct Task {
    int kind, w, v, c, g;
    bool own, lay;
};

// pair (row, index) of element e of a stage with R rows and `extra` strip pairs per row
__device__ __forceinline__ bool stage_pair(int e, int R, int extra, int *row, int *pair)
{
    if (e < 16 * R) { *row = e >> 4; *pair = e & 15; return true; }
    e -= 16 * R;
    if (e >= extra * R) return false;
    *row = extra == 2 ? e >> 1 : e;
    *pair = 16 + (extra == 2 ? (e & 1) : 0);
    return true;
}

__device__ __forceinline__ Task make_task(int phase, int tid, int i0, int j0, const TbArgs &P)
{
    Task k{0, 0, 0, 0, 0, false, false};
    int i = 0, j = 0, r, q;
    if (phase == 1) {
        if (tid < 224 && stage_pair(tid, 11, 2, &r, &q)) { k.kind = 1; i = i0 - 2 + 2 * q; j = j0 - 2 + r; }
        else if (tid >= 224 && stage_pair(tid - 224, 9, 1, &r, &q)) { k.kind = 3; i = i0 - 2 + 2 * q; j = j0 - 1 + r; }
    } else {
        if (tid < 192 && stage_pair(tid, 10, 2, &r, &q)) { k.kind = 2; i = i0 - 2 + 2 * q; j = j0 - 1 + r; }
        else if (tid >= 192 && stage_pair(tid - 192, 8, 0, &r, &q)) { k.kind = 4; i = i0 + 2 * q; j = j0 + r; }
    }
    if (!k.kind) return k;
    k.w = (j - j0 + 2) * WXN + (i - i0 + 4);
    k.v = (j - j0 + 2) * WXR + (i - i0 + 4);
    k.c = (j - j0 + 1) * CXN + (i - i0 + 16);
    k.g = j * P.px + i;
    k.own = i >= i0 && i + 1 < i0 + TBX && j >= j0 && j < j0 + TBY;
    k.lay = i == P.bx0 || i + 1 == P.bx1 || j == P.by0 || j == P.by1;
    return k;
}

__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
// a - b, exactly rounded (fused multiply-add by -1 rounds once)
__device__ __forceinline__ float2 dif(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// d1 r1 - d2 r2, with nr2 = -r2 (one rounding for the product d1 r1, one for the fused tail)
__device__ __forceinline__ float2 curl(float2 d1, float2 r1, float2 d2, float2 nr2)
{
    return __ffma2_rn(d2, nr2, __fmul2_rn(d1, r1));
}

struct Coef {
    float2 rx, ry, rz, nrx, nry, nrz, ndb;
};

// H update of a node pair (S1 from step-n data, S3 from E^{n+1}): e0/e1 = E on planes p, p+1,
// h0 = H on plane p, read at index w in rows of RS floats; result into the ring hw at index v
// A thread keeps its stage and pair on every plane, so the E_x, E_y (or H_x, H_y) of the
// pair that one plane reads as its upper (lower) z-neighbour are the next plane's centre
// values: they are carried in registers (cx, cy) once the stage has run on a plane before.
template <int RS>
__device__ __forceinline__ void h_pair(const float *e0, const float *e1, const float *h0, float *hw, int w,
                                       int v, const Coef &K, float2 &cx, float2 &cy, bool carried)
{
    constexpr int RN = RS * WYN;   // one component of a plane
    const float2 ex = carried ? cx : ld2(e0 + w), ey = carried ? cy : ld2(e0 + RN + w);
    const float2 ez = ld2(e0 + 2 * RN + w);
    const float2 exU = ld2(e0 + w + RS), ezU = ld2(e0 + 2 * RN + w + RS);
    const float2 eyR = make_float2(ey.y, e0[RN + w + 2]), ezR = make_float2(ez.y, e0[2 * RN + w + 2]);
    const float2 ex1 = ld2(e1 + w), ey1 = ld2(e1 + RN + w);
    cx = ex1;
    cy = ey1;
    // H_x -= dt/mu0 (dEz/dy - dEy/dz), H_y -= dt/mu0 (dEx/dz - dEz/dx), H_z -= dt/mu0 (dEy/dx - dEx/dy)
    st2(hw + v, __ffma2_rn(curl(dif(ezU, ez), K.ry, dif(ey1, ey), K.nrz), K.ndb, ld2(h0 + w)));
    st2(hw + WR + v, __ffma2_rn(curl(dif(ex1, ex), K.rz, dif(ezR, ez), K.nrx), K.ndb, ld2(h0 + RN + w)));
    st2(hw + 2 * WR + v, __ffma2_rn(curl(dif(eyR, ey), K.rx, dif(exU, ex), K.nry), K.ndb, ld2(h0 + 2 * RN + w)));
}

// E update of a node pair: eo = E before (index we in rows of ES floats), ha/hp = H on planes
// k, k-1 (ring index v), cl = class tile of plane k.  Class 0 (PEC) has Ca = Cb = 0, so its
// edges stay zero.
template <int ES>
__device__ __forceinline__ void e_pair(const float *eo, int we, const float *ha, const float *hp, int v,
                                       const unsigned char *cl, const float2 *CT, int c, const Coef &K, float2 *vx,
                                       float2 *vy, float2 *vz, float2 &cx, float2 &cy, bool carried)
{
    constexpr int EN = ES * WYN;
    const float2 hx = ld2(ha + v), hy = ld2(ha + WR + v), hz = ld2(ha + 2 * WR + v);
    const float2 hxD = ld2(ha + v - WXR), hzD = ld2(ha + 2 * WR + v - WXR);
    const float2 hyL = make_float2(ha[WR + v - 1], hy.x), hzL = make_float2(ha[2 * WR + v - 1], hz.x);
    const float2 hpx = carried ? cx : ld2(hp + v), hpy = carried ? cy : ld2(hp + WR + v);
    cx = hx;
    cy = hy;
    const unsigned cxx = *reinterpret_cast<const unsigned short *>(cl + c);
    const unsigned cyy = *reinterpret_cast<const unsigned short *>(cl + CN + c);
    const unsigned czz = *reinterpret_cast<const unsigned short *>(cl + 2 * CN + c);
    const float2 ax0 = CT[cxx & 255], ax1 = CT[cxx >> 8];
    const float2 ay0 = CT[cyy & 255], ay1 = CT[cyy >> 8];
    const float2 az0 = CT[czz & 255], az1 = CT[czz >> 8];
    // E_x = Ca E_x + Cb (dHz/dy - dHy/dz), E_y = Ca E_y + Cb (dHx/dz - dHz/dx),
    // E_z = Ca E_z + Cb (dHy/dx - dHx/dy)
    *vx = __ffma2_rn(make_float2(ax0.y, ax1.y), curl(dif(hz, hzD), K.ry, dif(hy, hpy), K.nrz),
                     __fmul2_rn(make_float2(ax0.x, ax1.x), ld2(eo + we)));
    *vy = __ffma2_rn(make_float2(ay0.y, ay1.y), curl(dif(hx, hpx), K.rz, dif(hz, hzL), K.nrx),
                     __fmul2_rn(make_float2(ay0.x, ay1.x), ld2(eo + EN + we)));
    *vz = __ffma2_rn(make_float2(az0.y, az1.y), curl(dif(hy, hyL), K.rx, dif(hx, hxD), K.nry),
                     __fmul2_rn(make_float2(az0.x, az1.x), ld2(eo + 2 * EN + we)));
}

__global__ void __launch_bounds__(TBN, 2)
k_yee_tb2(const BatchItem *items, const TbArgs *args, const CUtensorMap *maps, int phase_buf, int *status)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const BatchItem it = items[blockIdx.x];
    const TbArgs P = args[phase_buf];
    const CUtensorMap *tmW = maps + 2 * phase_buf, *tmC = maps + 2 * phase_buf + 1;
    const int tid = threadIdx.x;
    const int i0 = it.i0, j0 = it.j0, kb = it.kb, ke = it.ke;
    float2 *CT = reinterpret_cast<float2 *>(sm + CT_OFF);
    const uint32_t bar0 = smem_u32(sm + BAR_OFF);
    if (smem_u32(sm) & 127u) {
        if (tid == 0) atomicOr(status, 4);
        return;
    }
    if (tid == 0) {
        for (int s = 0; s < FST; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int q = tid; q < kMaxClasses; q += TBN) CT[q] = make_float2(P.ctab[2 * q], P.ctab[2 * q + 1]);
    __syncthreads();

    auto issue = [&](int p) {   // one thread: step-n plane p -> field stage p & 3, class slot p % 6
        unsigned char *st = sm + (p & 3) * 2 * PL;
        const uint32_t bar = bar0 + 8 * (p & 3);
        mbar_expect_tx(bar, TX_BYTES);
        tma_load_4d(smem_u32(st), tmW, i0 - 4, j0 - 2, p, 0, bar);
        tma_load_4d(smem_u32(st + PL), tmW, i0 - 4, j0 - 2, p, 3, bar);
        tma_load_4d(smem_u32(sm + C_OFF + (p % CSL) * CSLOT), tmC, i0 - 16, j0 - 1, p, 0, bar);
    };
    uint32_t ph = 0;   // thread 0: parity of each stage's next completion
    auto wait_plane = [&](int p) -> bool {
        bool ok = true;
        if (tid == 0) {
            const int s = p & 3;
            ok = mbar_wait(bar0 + 8 * s, (ph >> s) & 1u);
            ph ^= 1u << s;
        }
        return __syncthreads_and(ok);
    };
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(kb - 2);
        issue(kb - 1);
        issue(kb);
    }
    const Task T1 = make_task(1, tid, i0, j0, P), T2 = make_task(2, tid, i0, j0, P);
    if (!wait_plane(kb - 2)) {
        if (tid == 0) atomicOr(status, 2);
        return;
    }

    Coef K;
    K.rx = make_float2(P.rdx, P.rdx);
    K.ry = make_float2(P.rdy, P.rdy);
    K.rz = make_float2(P.rdz, P.rdz);
    K.nrx = make_float2(-P.rdx, -P.rdx);
    K.nry = make_float2(-P.rdy, -P.rdy);
    K.nrz = make_float2(-P.rdz, -P.rdz);
    K.ndb = make_float2(-P.db, -P.db);
    const int plane = (int)P.plane, npts = (int)P.npts;
    float *const HA = reinterpret_cast<float *>(sm + HA_OFF);
    float *const EA = reinterpret_cast<float *>(sm + EA_OFF);
    float *const HB = reinterpret_cast<float *>(sm + HB_OFF);
    const bool xy_edge = i0 == P.bx0 || i0 + TBX - 1 == P.bx1 || j0 == P.by0 || j0 + TBY - 1 == P.by1;
    // ring slots of plane q-1: a = (q-1) mod 3 (H^{n+1/2}, E^{n+1}), b = (q-1) mod 6 (classes)
    int a = (kb - 2) % 3, b = (kb - 2) % CSL;
    float2 c1x = make_float2(0.f, 0.f), c1y = c1x, c2x = c1x, c2y = c1x;   // carried z-neighbours

    for (int q = kb - 1; q <= ke + 3; ++q) {
        if (q <= ke + 2) {
            if (!wait_plane(q)) {
                if (tid == 0) atomicOr(status, 2);
                return;
            }
        } else {
            __syncthreads();
        }
        const int a1 = a == 2 ? 0 : a + 1, a2 = a == 0 ? 2 : a - 1;   // (q-3) mod 3, (q-2) mod 3
        const int p3 = q - 3;
        const float *f0 = reinterpret_cast<const float *>(sm + ((q - 1) & 3) * 2 * PL);   // step n, plane q-1
        const float *f1 = reinterpret_cast<const float *>(sm + (q & 3) * 2 * PL);         // step n, plane q
        float *haw = HA + a * 3 * WR;                 // H^{n+1/2} plane q-1
        const float *hap = HA + a2 * 3 * WR;          // plane q-2
        const float *ha3 = HA + a1 * 3 * WR;          // plane q-3
        float *eaw = EA + a * 3 * WR;                 // E^{n+1} plane q-1
        const float *ea3 = EA + a1 * 3 * WR, *ea2 = EA + a2 * 3 * WR;
        float *hb3 = HB + (p3 & 1) * 3 * WR;          // H^{n+3/2} plane q-3
        const float *hb4 = HB + ((p3 + 1) & 1) * 3 * WR;
        const unsigned char *cl1 = sm + C_OFF + b * CSLOT;
        const unsigned char *cl3 = sm + C_OFF + (b >= 2 ? b - 2 : b + 4) * CSLOT;

        // phase 1: S1 on plane q-1, S3 on plane q-3
        if (T1.kind == 1 && q <= ke + 2) h_pair<WXN>(f0, f1, f0 + 3 * WN, haw, T1.w, T1.v, K, c1x, c1y, q > kb - 1);
        if (T1.kind == 3 && q >= kb + 2) h_pair<WXR>(ea3, ea2, ha3, hb3, T1.v, T1.v, K, c1x, c1y, q > kb + 2);
        __syncthreads();
        // every thread finished plane q-2's stage and plane q-4's classes before this plane's
        // first barrier, and phase 2 reads neither: the last warp, which has no phase-2 task,
        // refills them with plane q+2
        if (tid == TBN - 32 && q <= ke) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(q + 2);
        }
        // phase 2: S2 on plane q-1, S4 on plane q-3 (into C)
        if (T2.kind == 2 && q >= kb && q <= ke + 2) {
            float2 vx, vy, vz;
            e_pair<WXN>(f0, T2.w, haw, hap, T2.v, cl1, CT, T2.c, K, &vx, &vy, &vz, c2x, c2y, q > kb);
            st2(eaw + T2.v, vx);
            st2(eaw + WR + T2.v, vy);
            st2(eaw + 2 * WR + T2.v, vz);
            // the box's outer node layer at n + 1 (and its H^{n+1/2}) for the frame's second
            // step; a pair with one layer node writes both (the other value is also correct)
            const int k = q - 1;
            if (T2.own && k >= kb && k <= ke && (k == P.bz0 || k == P.bz1 || (xy_edge && T2.lay))) {
                float *B = P.B + (k * plane + T2.g);
                st2(B, vx);
                st2(B + npts, vy);
                st2(B + 2 * npts, vz);
                st2(B + 3 * npts, ld2(haw + T2.v));
                st2(B + 4 * npts, ld2(haw + WR + T2.v));
                st2(B + 5 * npts, ld2(haw + 2 * WR + T2.v));
            }
        }
        if (T2.kind == 4 && q >= kb + 3) {
            float2 vx, vy, vz;
            e_pair<WXR>(ea3, T2.v, hb3, hb4, T2.v, cl3, CT, T2.c, K, &vx, &vy, &vz, c2x, c2y, q > kb + 3);
            float *C = P.C + (p3 * plane + T2.g);
            st2(C, vx);
            st2(C + npts, vy);
            st2(C + 2 * npts, vz);
            st2(C + 3 * npts, ld2(hb3 + T2.v));
            st2(C + 4 * npts, ld2(hb3 + WR + T2.v));
            st2(C + 5 * npts, ld2(hb3 + 2 * WR + T2.v));
        }
        a = a == 2 ? 0 : a + 1;
        b = b == CSL - 1 ? 0 : b + 1;
    }
}

}  // namespace

cudaError_t tb_prepare()
{
    return cudaFuncSetAttribute(k_yee_tb2, cudaFuncAttributeMaxDynamicSharedMemorySize, TB_BYTES);
}

cudaError_t launch_tb2(const BatchItem *items, int count, const TbArgs *args, const CUtensorMap *maps,
                       int phase, int *status, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_yee_tb2<<<count, TBN, TB_BYTES, s>>>(items, args, maps, phase, status);
    return cudaGetLastError();
}

}  // namespace yf
