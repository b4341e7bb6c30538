// Two-step (temporally blocked) Yee update of the inner box, FP32 (variant 4).
//
// The inner box is a set of whole 32 x TY tiles (TY = 8 or 16) and a z range that keep at least three nodes
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
// z is marched with the stages skewed by three planes, so that each plane iteration q has
// two phases and one block barrier between them: {S1 on plane q-1, S3 on plane q-4}, barrier,
// {S2 on plane q-1, S4 on plane q-4}.  Every value a phase reads was written before an
// earlier barrier, and every slot a phase overwrites was last read before one, so no barrier
// is needed between one iteration's second phase and the next iteration's first.  A thread
// runs S1 and S2 (or S3 and S4) on the same node pair: its own new H and its own old E pass
// between its two stages in registers.
//
// Step-n planes arrive by TMA two planes ahead, issued by an idle thread right after the
// barrier: the E window of 40 x (TY + 4) nodes and the H window of 40 x (TY + 3) (x from
// i0-4, y from j0-2) in four stages, and with plane p's fields the class tiles (80 x (TY + 2)
// bytes) of plane p-1, in six slots (S4 reads the classes of plane q-4).  Every thread waits
// on a stage's mbarrier itself.  H^{n+1/2} and E^{n+1} are kept for four planes and H^{n+3/2}
// for two, in rings of rows of 44 floats (a 12-bank shift per row spreads the strips of eight
// rows over all 32 banks) that hold only the rows each stage writes: TY + 3, TY + 2 and
// TY + 1.  TY = 8 takes 113 KB of shared memory (two blocks of 384 threads per SM), TY = 16
// 195 KB (one block of 672 threads), which recomputes 1.18 instead of 1.29 nodes per output
// node.
//
// The single-step frame advances the rest of the grid n -> n+1 (A -> B) and n+1 -> n+2
// (B -> C).  Its second step reads the box's outermost node layer at n + 1 from B (a window
// reaches one node into the box), so this kernel also writes E^{n+1} and H^{n+1/2} of that
// layer into B.  Every mbarrier wait is bounded; a thread whose wait gives up carries on (its
// shared-memory reads stay in bounds), the block leaves together at the next barrier, sets
// bit 1 of the status word, and the issuing thread first waits, again bounded, for the copies
// it has in flight.  The host side (box, work items, arguments, the pair of steps) is in
// yf_tb_plan.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "yf_internal.h"

namespace yf {
namespace {

constexpr int TBX = kTbTileX;                        // output tile width
// windows: x from i0-4, 40 wide; rings: rows of 44 floats (a 12-bank shift per row spreads
// the strips of eight rows over all 32 banks); class tiles: x from i0-16, 80 bytes wide
constexpr int WXN = kTbWinX, WXR = 44, CXN = kTbClsX;
constexpr int FST = 4, CSL = 6;                      // field stages, class slots

// Layout of a block whose output tile is 32 x TY nodes (TY = 8: two blocks per SM; TY = 16:
// one).  Group A (S1, S2) works on rows j0-2..j0+TY, group B (S3, S4) on rows j0-1..j0+TY-1.
template <int TY>
struct TbShape {
    static constexpr int RA = TY + 3, RB = TY + 1;                 // rows of groups A and B
    static constexpr int NA = 18 * RA, NB = 17 * RB;               // their threads (pairs)
    static constexpr int BBASE = (NA + 31) / 32 * 32;              // group B's first thread
    static constexpr int TBN = BBASE + (NB + 31) / 32 * 32;        // block
    static constexpr int ISSUER = BBASE - 1;                       // idle: BBASE > NA
    static constexpr int WYN = TY + 4, WYH = TY + 3, CYN = TY + 2; // window / class-tile rows
    static constexpr int WN = WXN * WYN, WNH = WXN * WYH, CN = CXN * CYN;
    // rings: H^{n+1/2} rows j0-2..j0+TY, E^{n+1} rows j0-1..j0+TY, H^{n+3/2} j0-1..j0+TY-1
    static constexpr int RHA = WXR * (TY + 3), REA = WXR * (TY + 2), RHB = WXR * (TY + 1);
    static constexpr int CSLOT = (3 * CN + 127) / 128 * 128;       // one class slot (bytes)
    static constexpr int PLE = 3 * WN * 4;                         // E window of a stage (bytes)
    static constexpr int PLH = (3 * WNH * 4 + 127) / 128 * 128;    // H window of a stage (bytes)
    static constexpr int SST = (PLE + 127) / 128 * 128 + PLH;      // one stage
    static constexpr int PLE_PAD = SST - PLH;
    static constexpr int C_OFF = FST * SST;
    static constexpr int HA_OFF = C_OFF + CSL * CSLOT;             // H^{n+1/2} [4][3][RHA]
    static constexpr int EA_OFF = HA_OFF + 4 * 3 * RHA * 4;        // E^{n+1}   [4][3][REA]
    static constexpr int HB_OFF = EA_OFF + 4 * 3 * REA * 4;        // H^{n+3/2} [2][3][RHB]
    static constexpr int CT_OFF = HB_OFF + 2 * 3 * RHB * 4;        // (Ca, Cb) per class
    static constexpr int BAR_OFF = CT_OFF + 2 * kMaxClasses * 4;
    static constexpr int BYTES = BAR_OFF + 8 * FST;
    static constexpr uint32_t TX_BYTES = 3 * WN * 4 + 3 * WNH * 4 + 3 * CN;
    static constexpr int BLOCKS_PER_SM = TY == 8 ? 2 : 1;
    static_assert(NA < BBASE, "an idle thread issues the refills");
    static_assert(SST % 128 == 0 && C_OFF % 128 == 0 && CSLOT % 128 == 0 && PLE_PAD % 128 == 0,
                  "TMA destinations 128-byte aligned");
    static_assert(HA_OFF % 16 == 0 && EA_OFF % 16 == 0 && HB_OFF % 16 == 0, "ring planes 16-byte aligned");
    static_assert(BLOCKS_PER_SM * (BYTES + 1024) <= 228 * 1024, "shared memory per SM");
};

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

// Each thread updates one pair of x-adjacent nodes (i, i+1), i - i0 even, in both half steps
// of one time step: group A runs S1 (phase 1) and S2 (phase 2), group B runs S3 and S4, each
// on the same pair of nodes.  A half-warp takes the first 16 pairs of one row (128 contiguous
// bytes, no bank conflicts); the one or two pairs left at the right end of each row form
// short strips:
//   group A: rows j0-2..j0+TY: 16 (TY + 3) threads on pairs 0..15 from i0-2, then 2 (TY + 3)
//            strip threads on pairs 16, 17 (S1 on every row, S2 on rows j0-1..j0+TY)
//   group B: from the next warp, rows j0-1..j0+TY-1: 16 (TY + 1) threads on pairs 0..15
//            from i0-2, then TY + 1 strip threads on pair 16 (S3 on every row, S4 on rows
//            j0..j0+TY-1 and pairs from i0)
// (TY = 8: group A threads 0..197, group B 224..376, 384 threads.)
// Pairs reach one node past the needed ranges on the left of S2 and S3 and on the right of
// S1 and S2; those extra nodes read neighbours nobody computed and feed nothing.  The pair's
// values move as float2 (64-bit shared loads, one 32-bit load for the neighbour shifted by
// one node in x) through Blackwell's paired FP32 arithmetic.
// kind: 1 group A, 3 group B, 0 idle; e: the E stage runs on this pair; w: index of the pair's
// first node in the windows; vh, ve, vb: in the H^{n+1/2}, E^{n+1} and H^{n+3/2} rings; c: in
// the class tile; g: its offset j px + i in a field plane; own: the pair is in the block's
// tile; lay: a node of it lies on the box's outer layer in x or y.
struct Task {
    int kind, w, vh, ve, vb, c, g;
    bool e, own, lay;
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

template <int TY>
__device__ __forceinline__ Task make_task(int tid, int i0, int j0, const TbArgs &P)
{
    using S = TbShape<TY>;
    Task k{0, 0, 0, 0, 0, 0, 0, false, false, false};
    int i = 0, j = 0, r, q;
    if (tid < S::BBASE && stage_pair(tid, S::RA, 2, &r, &q)) {
        k.kind = 1;
        k.e = r >= 1;
        i = i0 - 2 + 2 * q;
        j = j0 - 2 + r;
    } else if (tid >= S::BBASE && stage_pair(tid - S::BBASE, S::RB, 1, &r, &q)) {
        k.kind = 3;
        k.e = r >= 1 && q >= 1;
        i = i0 - 2 + 2 * q;
        j = j0 - 1 + r;
    }
    if (!k.kind) return k;
    k.w = (j - j0 + 2) * WXN + (i - i0 + 4);
    k.vh = (j - j0 + 2) * WXR + (i - i0 + 4);
    k.ve = k.vh - WXR;
    k.vb = k.ve;
    k.c = (j - j0 + 1) * CXN + (i - i0 + 16);
    k.g = j * P.px + i;
    k.own = i >= i0 && i + 1 < i0 + TBX && j >= j0 && j < j0 + TY;
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

// The pair's three components (E or H) held in registers between a thread's two stages.
struct Vec3 {
    float2 x, y, z;
};

// H update of a node pair (S1 from step-n data, S3 from E^{n+1}): e0/e1 = E on planes p, p+1
// (rows of ES floats, components EC apart, index w), h0 = H on plane p (components HC apart,
// index wh); result into the ring hw (components OC apart, index v) for the neighbours and
// into hn for the thread's own E stage, the pair's E on plane p into eo.  A thread keeps its
// pair on every plane, so the E_x, E_y of the pair that one plane reads as its upper
// z-neighbour are the next plane's centre values: they are carried in registers (cx, cy) once
// the stage has run on a plane before.
template <int ES, int EC, int HC, int OC>
__device__ __forceinline__ void h_pair(const float *e0, const float *e1, int w, const float *h0, int wh,
                                       float *hw, int v, const Coef &K, float2 &cx, float2 &cy, bool carried,
                                       Vec3 &eo, Vec3 &hn)
{
    const float2 ex = carried ? cx : ld2(e0 + w), ey = carried ? cy : ld2(e0 + EC + w);
    const float2 ez = ld2(e0 + 2 * EC + w);
    const float2 exU = ld2(e0 + w + ES), ezU = ld2(e0 + 2 * EC + w + ES);
    const float2 eyR = make_float2(ey.y, e0[EC + w + 2]), ezR = make_float2(ez.y, e0[2 * EC + w + 2]);
    const float2 ex1 = ld2(e1 + w), ey1 = ld2(e1 + EC + w);
    cx = ex1;
    cy = ey1;
    eo.x = ex;
    eo.y = ey;
    eo.z = ez;
    // H_x -= dt/mu0 (dEz/dy - dEy/dz), H_y -= dt/mu0 (dEx/dz - dEz/dx), H_z -= dt/mu0 (dEy/dx - dEx/dy)
    hn.x = __ffma2_rn(curl(dif(ezU, ez), K.ry, dif(ey1, ey), K.nrz), K.ndb, ld2(h0 + wh));
    hn.y = __ffma2_rn(curl(dif(ex1, ex), K.rz, dif(ezR, ez), K.nrx), K.ndb, ld2(h0 + HC + wh));
    hn.z = __ffma2_rn(curl(dif(eyR, ey), K.rx, dif(exU, ex), K.nry), K.ndb, ld2(h0 + 2 * HC + wh));
    st2(hw + v, hn.x);
    st2(hw + OC + v, hn.y);
    st2(hw + 2 * OC + v, hn.z);
}

// E update of a node pair from registers and a ring: h = the pair's H on plane k (the
// thread's own H stage), ha = the ring of plane k (components HC apart, index v) for the y-
// and x-neighbours, hpx/hpy = the pair's H_x, H_y on plane k-1 (the own H stage one plane
// earlier), eo = the pair's E before the update, cl = class tile of plane k.  Class 0 (PEC)
// has Ca = Cb = 0, so its edges stay zero; its three components are CN bytes apart.
template <int HC, int CN>
__device__ __forceinline__ void e_pair(const Vec3 &h, const float *ha, int v, float2 hpx, float2 hpy,
                                       const Vec3 &eo, const unsigned char *cl, const float2 *CT, int c,
                                       const Coef &K, float2 *vx, float2 *vy, float2 *vz)
{
    const float2 hx = h.x, hy = h.y, hz = h.z;
    const float2 hxD = ld2(ha + v - WXR), hzD = ld2(ha + 2 * HC + v - WXR);
    const float2 hyL = make_float2(ha[HC + v - 1], hy.x), hzL = make_float2(ha[2 * HC + v - 1], hz.x);
    const unsigned cxx = *reinterpret_cast<const unsigned short *>(cl + c);
    const unsigned cyy = *reinterpret_cast<const unsigned short *>(cl + CN + c);
    const unsigned czz = *reinterpret_cast<const unsigned short *>(cl + 2 * CN + c);
    const float2 ax0 = CT[cxx & 255], ax1 = CT[cxx >> 8];
    const float2 ay0 = CT[cyy & 255], ay1 = CT[cyy >> 8];
    const float2 az0 = CT[czz & 255], az1 = CT[czz >> 8];
    // E_x = Ca E_x + Cb (dHz/dy - dHy/dz), E_y = Ca E_y + Cb (dHx/dz - dHz/dx),
    // E_z = Ca E_z + Cb (dHy/dx - dHx/dy)
    *vx = __ffma2_rn(make_float2(ax0.y, ax1.y), curl(dif(hz, hzD), K.ry, dif(hy, hpy), K.nrz),
                     __fmul2_rn(make_float2(ax0.x, ax1.x), eo.x));
    *vy = __ffma2_rn(make_float2(ay0.y, ay1.y), curl(dif(hx, hpx), K.rz, dif(hz, hzL), K.nrx),
                     __fmul2_rn(make_float2(ay0.x, ay1.x), eo.y));
    *vz = __ffma2_rn(make_float2(az0.y, az1.y), curl(dif(hy, hyL), K.rx, dif(hx, hxD), K.nry),
                     __fmul2_rn(make_float2(az0.x, az1.x), eo.z));
}

template <int TY>
__global__ void __launch_bounds__(TbShape<TY>::TBN, TbShape<TY>::BLOCKS_PER_SM)
k_yee_tb2(const BatchItem *items, const TbArgs *args, const CUtensorMap *maps, int phase_buf, int *status)
{
    using S = TbShape<TY>;
    constexpr int TBN = S::TBN, ISSUER = S::ISSUER, SST = S::SST, CSLOT = S::CSLOT;
    constexpr int WN = S::WN, WNH = S::WNH, RHA = S::RHA, REA = S::REA, RHB = S::RHB;
    extern __shared__ __align__(128) unsigned char sm[];
    const BatchItem it = items[blockIdx.x];
    // the item's grid: its three argument sets and nine maps (one grid: inst = 0)
    const TbArgs P = args[3 * it.inst + phase_buf];
    const CUtensorMap *tmE = maps + 3 * (3 * it.inst + phase_buf), *tmH = tmE + 1, *tmC = tmE + 2;
    const int tid = threadIdx.x;
    const int i0 = it.i0, j0 = it.j0, kb = it.kb, ke = it.ke;
    float2 *CT = reinterpret_cast<float2 *>(sm + S::CT_OFF);
    const uint32_t bar0 = smem_u32(sm + S::BAR_OFF);
    if (smem_u32(sm) & 127u) {
        if (tid == 0) atomicOr(status, 4);
        return;
    }
    if (tid == ISSUER) {
        for (int s = 0; s < FST; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int q = tid; q < kMaxClasses; q += TBN) CT[q] = make_float2(P.ctab[2 * q], P.ctab[2 * q + 1]);
    __syncthreads();

    // one thread: step-n plane p -> field stage p & 3 (E and H windows), and the class tiles of
    // plane p - 1 -> slot (p - 1) mod 6, all on the stage's mbarrier (p >= kb - 2 >= -2; planes
    // below the grid, for a box on the ground, arrive as zeros)
    auto issue = [&](int p) {
        unsigned char *st = sm + (p & 3) * SST;
        const uint32_t bar = bar0 + 8 * (p & 3);
        mbar_expect_tx(bar, S::TX_BYTES);
        tma_load_4d(smem_u32(st), tmE, i0 - 4, j0 - 2, p, 0, bar);
        tma_load_4d(smem_u32(st + S::PLE_PAD), tmH, i0 - 4, j0 - 2, p, 3, bar);
        tma_load_4d(smem_u32(sm + S::C_OFF + ((p + CSL - 1) % CSL) * CSLOT), tmC, i0 - 16, j0 - 1, p - 1, 0, bar);
    };
    // every thread waits for each plane itself, once, in plane order; ph holds the parity of
    // each stage's next completion
    uint32_t ph = 0;
    auto wait_plane = [&](int p) -> bool {
        const int s = p & 3;
        const bool ok = mbar_wait(bar0 + 8 * s, (ph >> s) & 1u);
        ph ^= 1u << s;
        return ok;
    };
    if (tid == ISSUER) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(kb - 2);
        issue(kb - 1);
        issue(kb);
    }
    const Task T = make_task<TY>(tid, i0, j0, P);
    bool bad = !wait_plane(kb - 2);

    Coef K;
    K.rx = make_float2(P.rdx, P.rdx);
    K.ry = make_float2(P.rdy, P.rdy);
    K.rz = make_float2(P.rdz, P.rdz);
    K.nrx = make_float2(-P.rdx, -P.rdx);
    K.nry = make_float2(-P.rdy, -P.rdy);
    K.nrz = make_float2(-P.rdz, -P.rdz);
    K.ndb = make_float2(-P.db, -P.db);
    const int plane = (int)P.plane, npts = (int)P.npts;
    float *const HA = reinterpret_cast<float *>(sm + S::HA_OFF);
    float *const EA = reinterpret_cast<float *>(sm + S::EA_OFF);
    float *const HB = reinterpret_cast<float *>(sm + S::HB_OFF);
    const bool xy_edge = i0 == P.bx0 || i0 + TBX - 1 == P.bx1 || j0 == P.by0 || j0 + TY - 1 == P.by1;
    int b = (kb - 2 + CSL) % CSL;   // class slot of plane q-1 (kb >= 0)
    // carried z-neighbours: the E_x, E_y the H stage reads on the plane above (the next
    // plane's centre values), and the H_x, H_y the thread's H stage produced on the previous
    // plane (the E stage's lower z-neighbour)
    float2 c1x = make_float2(0.f, 0.f), c1y = c1x, c2x = c1x, c2y = c1x;
    Vec3 eo, hn;   // the pair's E before and H after the H stage, kept for its E stage

    for (int q = kb - 1; q <= ke + 4; ++q) {
        bool wok = true;
        if (q <= ke + 2) {
            wok = wait_plane(q);
            bad = bad || !wok;
        }
        const unsigned char *s0 = sm + ((q - 1) & 3) * SST, *s1 = sm + (q & 3) * SST;
        const float *f0 = reinterpret_cast<const float *>(s0);          // step n: E, plane q-1
        const float *f1 = reinterpret_cast<const float *>(s1);          //         E, plane q
        const float *g0 = reinterpret_cast<const float *>(s0 + S::PLE_PAD);   //   H, plane q-1
        float *haw = HA + ((q - 1) & 3) * 3 * RHA;           // H^{n+1/2} plane q-1
        const float *ha4 = HA + (q & 3) * 3 * RHA;           //           plane q-4
        float *eaw = EA + ((q - 1) & 3) * 3 * REA;           // E^{n+1}   plane q-1
        const float *ea4 = EA + (q & 3) * 3 * REA;           //           plane q-4
        const float *ea3 = EA + ((q + 1) & 3) * 3 * REA;     //           plane q-3
        float *hb4 = HB + (q & 1) * 3 * RHB;                 // H^{n+3/2} plane q-4
        const unsigned char *cl1 = sm + S::C_OFF + b * CSLOT;                          // classes, plane q-1
        const unsigned char *cl4 = sm + S::C_OFF + (b >= 3 ? b - 3 : b + 3) * CSLOT;   //          plane q-4
        const int p4 = q - 4;

        // phase 1: S1 on plane q-1 (group A), S3 on plane q-4 (group B)
        const bool hstage = T.kind == 1 ? q <= ke + 2 : (T.kind == 3 && q >= kb + 3);
        if (T.kind == 1 && hstage)
            h_pair<WXN, WN, WNH, RHA>(f0, f1, T.w, g0, T.w, haw, T.vh, K, c1x, c1y, q > kb - 1, eo, hn);
        if (T.kind == 3 && hstage)
            h_pair<WXR, REA, RHA, RHB>(ea4, ea3, T.ve, ha4, T.vh, hb4, T.vb, K, c1x, c1y, q > kb + 3, eo, hn);
        if (__syncthreads_or(bad)) {
            if (tid == ISSUER) {
                // the copies still in flight: plane q+1, and plane q if this thread's own wait
                // for it gave up
                if (q + 1 <= ke + 2) mbar_wait(bar0 + 8 * ((q + 1) & 3), (ph >> ((q + 1) & 3)) & 1u);
                if (!wok) mbar_wait(bar0 + 8 * (q & 3), ((ph >> (q & 3)) & 1u) ^ 1u);
                atomicOr(status, 2);
            }
            return;
        }
        // every thread finished plane q-2's stage (last read in phase 1 of iteration q-1) and
        // plane q-5's classes (phase 2 of iteration q-1) before this barrier: refill them
        if (tid == ISSUER && q <= ke) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(q + 2);
        }
        // phase 2: S2 on plane q-1, S4 on plane q-4 (into C); the lower z-neighbour H of the
        // pair is the thread's own H stage of the previous plane (c2x, c2y)
        if (T.kind == 1 && T.e && q >= kb && q <= ke + 2) {
            float2 vx, vy, vz;
            e_pair<RHA, S::CN>(hn, haw, T.vh, c2x, c2y, eo, cl1, CT, T.c, K, &vx, &vy, &vz);
            st2(eaw + T.ve, vx);
            st2(eaw + REA + T.ve, vy);
            st2(eaw + 2 * REA + T.ve, vz);
            // the box's outer node layer at n + 1 (and its H^{n+1/2}) for the frame's second
            // step; a pair with one layer node writes both (the other value is also correct)
            const int k = q - 1;
            if (T.own && k >= kb && k <= ke && (k == P.bz0 || k == P.bz1 || (xy_edge && T.lay))) {
                float *B = P.B + (k * plane + T.g);
                st2(B, vx);
                st2(B + npts, vy);
                st2(B + 2 * npts, vz);
                st2(B + 3 * npts, hn.x);
                st2(B + 4 * npts, hn.y);
                st2(B + 5 * npts, hn.z);
            }
        }
        if (T.kind == 3 && T.e && q >= kb + 4) {
            float2 vx, vy, vz;
            e_pair<RHB, S::CN>(hn, hb4, T.vb, c2x, c2y, eo, cl4, CT, T.c, K, &vx, &vy, &vz);
            float *C = P.C + (p4 * plane + T.g);
            st2(C, vx);
            st2(C + npts, vy);
            st2(C + 2 * npts, vz);
            st2(C + 3 * npts, hn.x);
            st2(C + 4 * npts, hn.y);
            st2(C + 5 * npts, hn.z);
        }
        if (hstage) {
            c2x = hn.x;
            c2y = hn.y;
        }
        b = b == CSL - 1 ? 0 : b + 1;
    }
}

}  // namespace

cudaError_t tb_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_yee_tb2<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TbShape<8>::BYTES);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_yee_tb2<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, TbShape<16>::BYTES);
}

cudaError_t launch_tb2(const BatchItem *items, int count, const TbArgs *args, const CUtensorMap *maps,
                       int phase, int *status, cudaStream_t s, int tile_y)
{
    if (count <= 0) return cudaSuccess;
    if (tile_y == 16)
        k_yee_tb2<16><<<count, TbShape<16>::TBN, TbShape<16>::BYTES, s>>>(items, args, maps, phase, status);
    else
        k_yee_tb2<8><<<count, TbShape<8>::TBN, TbShape<8>::BYTES, s>>>(items, args, maps, phase, status);
    return cudaGetLastError();
}

}  // namespace yf
