// Host side of the two-step inner-box update (variant 4, FP32): the box, the three work
// lists (whole-grid single step, frame single step, two-step box items), their arguments and
// tensor maps, and the pair of steps with its stream structure.  The kernel is in yf_tb.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "yf_grid.h"
#include "yf_internal.h"

namespace yf {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// The box.  A two-step block over tile (i0, j0) and planes kb..ke reads step-n nodes
// i in [i0-2, i0+34], j in [j0-2, j0+9], k in [kb-2, ke+2] and recomputes H and E on most of
// them (the values at i0+33 and i0+34 only feed nodes nobody uses); the nodes it needs must
// see the plain update only.  So the box keeps three nodes from every
// absorbing slab and domain wall on the low sides and two (x, y) or three (z) on the high
// sides, except that it reaches down to a PEC wall at z = 0 (the ground): there the planes it
// reads below the grid arrive as zeros, which is what the wall's edges hold, and its stores
// stay in the grid.  Tiles whose x range widened by four nodes holds the source plane or a port plane
// are left out (the port epilogue reads and the source writes the frame's fields between
// the two steps).  x: the longest run of admissible 32-node tile columns; y: rows aligned to
// the frame's tile height; z: every admissible plane.  Returns false when no box fits.
}  // namespace

bool choose_box(const yf_grid *g, int box[6])
{
    const int n = g->pml_n;
    const int XL = g->pml_lo[0] ? n : 0, XH = g->pml_hi[0] ? g->nx - n : g->nx;
    const int YL = g->pml_lo[1] ? n : 0, YH = g->pml_hi[1] ? g->ny - n : g->ny;
    const int ZL = g->pml_lo[2] ? n : 0, ZH = g->pml_hi[2] ? g->nz - n : g->nz;
    std::vector<int> special;
    if (g->has_src) special.push_back(g->src_plane);
    for (const PortDev &d : g->ports) special.push_back(d.plane);
    const int ntx = g->nx / 32;
    int best = 0, bt0 = 0, run = 0;
    for (int tx = 0; tx < ntx; ++tx) {
        const int i0 = 32 * tx;
        bool ok = i0 - 3 >= XL && i0 + 34 <= XH;
        for (int s : special) ok = ok && !(s >= i0 - 4 && s <= i0 + 35);
        run = ok ? run + 1 : 0;
        if (run > best) { best = run; bt0 = tx - run + 1; }
    }
    const int A = std::max(g->box_ty, g->tile_y);
    const int by0 = (YL + 3 + A - 1) / A * A, byE = (YH - 2) / A * A;
    const int bz0 = g->pml_lo[2] ? ZL + 3 : 0, bz1 = ZH - 3;
    if (best < 1 || byE <= by0 || bz1 - bz0 + 1 < 4) return false;
    box[0] = 32 * bt0;
    box[1] = 32 * (bt0 + best) - 1;
    box[2] = by0;
    box[3] = byE - 1;
    box[4] = bz0;
    box[5] = bz1;
    return true;
}

namespace {

yf_status upload_items(const std::vector<BatchItem> items[5], TmaPlan *pl)
{
    std::vector<BatchItem> all;
    for (int k = 0; k < 5; ++k) {
        pl->offset[k] = (int)all.size();
        pl->count[k] = (int)items[k].size();
        all.insert(all.end(), items[k].begin(), items[k].end());
    }
    YF_CUDA_TRY(cudaMalloc(&pl->items, std::max<size_t>(1, all.size()) * sizeof(BatchItem)));
    if (!all.empty())
        YF_CUDA_TRY(cudaMemcpy(pl->items, all.data(), all.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    return YF_OK;
}

int kinds_used(const TmaPlan &pl)
{
    int k = 0;
    for (int q = 0; q < 5; ++q) k += pl.count[q] > 0;
    return k;
}

}  // namespace

void tb_free(yf_grid *g)
{
    TbPlan *t = g->tb;
    if (!t) return;
    if (t->stream) cudaStreamSynchronize(t->stream);
    cudaFree(t->full.items);
    cudaFree(t->full.args);
    cudaFree(t->full.maps);
    cudaFree(t->frame.items);
    cudaFree(t->items);
    cudaFree(t->args);
    cudaFree(t->maps);
    if (t->pstream) cudaStreamSynchronize(t->pstream);
    if (t->fork) cudaEventDestroy(t->fork);
    if (t->fork_next) cudaEventDestroy(t->fork_next);
    if (t->join) cudaEventDestroy(t->join);
    if (t->ev_src) cudaEventDestroy(t->ev_src);
    if (t->ev_p1) cudaEventDestroy(t->ev_p1);
    for (int q = 0; q < 2; ++q)
        if (t->ev_p2[q]) cudaEventDestroy(t->ev_p2[q]);
    if (t->stream) cudaStreamDestroy(t->stream);
    if (t->pstream) cudaStreamDestroy(t->pstream);
    delete t;
    g->tb = nullptr;
}

// The work items of grid `inst`, appended: the one-step items over the whole grid (full; the
// all-CPML kind in segments of at most mixed_seg planes, 0: whole), those outside the box
// (frame: items that straddle it in z keep their parts below and above it), and the two-step
// box items (tiles of 32 x ty over z segments of seg planes).
void tb_items(const yf_grid *g, int inst, bool have_box, const int B[6], int ty, int seg,
              std::vector<BatchItem> full[5], std::vector<BatchItem> frame[5], std::vector<BatchItem> &two,
              int mixed_seg)
{
    std::vector<BatchItem> own[5];   // this grid's items only: the vectors may hold other grids'
    tma_items(inst, g->nx, g->ny, g->nz, g->kseg, g->tile_y, g->pml_n, g->pml_lo, g->pml_hi, own, mixed_seg);
    for (int k = 0; k < 5; ++k) full[k].insert(full[k].end(), own[k].begin(), own[k].end());
    for (int k = 0; k < 5; ++k)
        for (const BatchItem &it : own[k]) {
            const bool inxy = have_box && it.i0 >= B[0] && it.i0 <= B[1] && it.j0 >= B[2] && it.j0 <= B[3];
            if (!inxy || it.ke < B[4] || it.kb > B[5]) {
                frame[k].push_back(it);
                continue;
            }
            if (it.kb < B[4]) frame[k].push_back(BatchItem{inst, it.i0, it.j0, it.kb, B[4] - 1});
            if (it.ke > B[5]) frame[k].push_back(BatchItem{inst, it.i0, it.j0, B[5] + 1, it.ke});
        }
    if (have_box)
        for (int kb = B[4]; kb <= B[5]; kb += seg)
            for (int j0 = B[2]; j0 <= B[3]; j0 += ty)
                for (int i0 = B[0]; i0 <= B[1]; i0 += kTbTileX)
                    two.push_back(BatchItem{inst, i0, j0, kb, std::min(B[5], kb + seg - 1)});
}

// The one-step arguments and maps of a grid with three buffers, by slot 2 * src + hpar (the
// step reads buffer src and writes the next one)
void tb_step_args(yf_grid *g, FusedArgs<float> fa[6], CUtensorMap fm[12])
{
    const int c0 = g->cur, h0 = g->hpar;
    for (int r = 0; r < 3; ++r)
        for (int h = 0; h < 2; ++h) {
            g->cur = r;
            g->hpar = h;
            fa[2 * r + h] = fused_args<float>(g);
            fm[2 * (2 * r + h)] = g->tmF[r];
            fm[2 * (2 * r + h) + 1] = g->tmC;
        }
    g->cur = c0;
    g->hpar = h0;
}

// The two-step arguments and maps of a grid by source buffer r (B = buffer r+1, C = r+2): the
// E window map, the H window map and the class-tile map of each
yf_status tb_box_args(yf_grid *g, const int B[6], int ty, TbArgs ta[3], CUtensorMap tm[9])
{
    PFN_cuTensorMapEncodeTiled_v12000 encode = encoder();
    if (!encode) return fail(YF_E_CUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t gdim[4] = {(cuuint64_t)g->px, (cuuint64_t)(g->ny + 1), (cuuint64_t)(g->nz + 1), 6};
    const cuuint64_t gstr[3] = {(cuuint64_t)g->px * 4, (cuuint64_t)g->plane * 4, (cuuint64_t)g->npts * 4};
    const cuuint32_t wbox[4] = {kTbWinX, (cuuint32_t)ty + 4, 1, 3};
    const cuuint32_t hbox[4] = {kTbWinX, (cuuint32_t)ty + 3, 1, 3};
    const cuuint64_t cdim[4] = {(cuuint64_t)g->px, (cuuint64_t)(g->ny + 1), (cuuint64_t)(g->nz + 1), 3};
    const cuuint64_t cstr[3] = {(cuuint64_t)g->px, (cuuint64_t)g->plane, (cuuint64_t)g->npts};
    const cuuint32_t cbox[4] = {kTbClsX, (cuuint32_t)ty + 2, 1, 3};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    for (int r = 0; r < 3; ++r) {
        TbArgs &a = ta[r];
        a.px = g->px;
        a.plane = g->plane;
        a.npts = g->npts;
        a.rdx = (float)(1.0 / g->dx);
        a.rdy = (float)(1.0 / g->dy);
        a.rdz = (float)(1.0 / g->dz);
        a.db = (float)(g->dt / kMu0);
        a.ctab = (const float *)g->ctab;
        a.B = (float *)g->buf[(r + 1) % 3];
        a.C = (float *)g->buf[(r + 2) % 3];
        a.bx0 = B[0]; a.bx1 = B[1]; a.by0 = B[2]; a.by1 = B[3]; a.bz0 = B[4]; a.bz1 = B[5];
        CUresult cr = encode(&tm[3 * r], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->buf[r], gdim, gstr, wbox, one,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr == CUDA_SUCCESS)
            cr = encode(&tm[3 * r + 1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->buf[r], gdim, gstr, hbox, one,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr == CUDA_SUCCESS)
            cr = encode(&tm[3 * r + 2], CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, g->cls_base, cdim, cstr, cbox, one,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return fail(YF_E_CUDA, "variant 4: tensor map encoding failed (%d)", (int)cr);
    }
    return YF_OK;
}

// Plan of variant 4 on a finalised FP32 grid whose three field buffers exist and whose field
// maps (tmF[0..2], tmC) are encoded for the grid's tile height.
yf_status tb_build(yf_grid *g)
{
    if (g->tb) return YF_OK;
    if (g->prec != YF_FP32) return fail(YF_E_INVALID, "variant 4 needs FP32 fields");
    if (!g->buf[2]) return fail(YF_E_STATE, "variant 4: third field buffer missing");
    // the two-step kernel indexes a buffer's six components with 32-bit offsets
    if (6 * g->npts > 2147483647L)
        return fail(YF_E_INVALID, "variant 4 needs 6 (nz+1)(ny+1) px < 2^31 (grid has %ld points)", g->npts);
    PFN_cuTensorMapEncodeTiled_v12000 encode = encoder();
    if (!encode) return fail(YF_E_CUDA, "cuTensorMapEncodeTiled is not available");
    TbPlan *t = new TbPlan();
    g->tb = t;
    auto bail = [&](yf_status st) { tb_free(g); return st; };

    std::vector<BatchItem> full[5], frame[5], two;
    t->ty = g->box_ty;
    const bool have_box = choose_box(g, t->box);
    const int *B = t->box;
    // z-planes per two-step block: as set by yf_set_box_shape, else twice the one-step
    // segment (the two-step block re-reads four halo planes instead of two); its rings are
    // indexed modulo their depth, so any length works
    tb_items(g, 0, have_box, B, t->ty, g->box_seg > 0 ? g->box_seg : 2 * g->kseg, full, frame, two);
    yf_status st;
    if ((st = upload_items(full, &t->full)) != YF_OK) return bail(st);
    if ((st = upload_items(frame, &t->frame)) != YF_OK) return bail(st);
    t->count = (int)two.size();
    if (cudaMalloc(&t->items, std::max<size_t>(1, two.size()) * sizeof(BatchItem)) != cudaSuccess ||
        (!two.empty() && cudaMemcpy(t->items, two.data(), two.size() * sizeof(BatchItem),
                                    cudaMemcpyHostToDevice) != cudaSuccess))
        return bail(fail(YF_E_OOM, "variant 4: work items"));

    std::vector<FusedArgs<float>> fa(6);
    std::vector<CUtensorMap> fm(12);
    tb_step_args(g, fa.data(), fm.data());
    if (cudaMalloc(&t->full.args, fa.size() * sizeof(FusedArgs<float>)) != cudaSuccess ||
        cudaMemcpy(t->full.args, fa.data(), fa.size() * sizeof(FusedArgs<float>), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc(&t->full.maps, fm.size() * sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMemcpy(t->full.maps, fm.data(), fm.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(YF_E_OOM, "variant 4: step arguments"));
    t->full.stride = t->frame.stride = 6;
    t->frame.args = t->full.args;
    t->frame.maps = t->full.maps;

    TbArgs ta[3];
    CUtensorMap tm[9];
    if ((st = tb_box_args(g, B, t->ty, ta, tm)) != YF_OK) return bail(st);
    if (cudaMalloc(&t->args, sizeof(ta)) != cudaSuccess ||
        cudaMemcpy(t->args, ta, sizeof(ta), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc(&t->maps, sizeof(tm)) != cudaSuccess ||
        cudaMemcpy(t->maps, tm, sizeof(tm), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(YF_E_OOM, "variant 4: two-step arguments"));
    if (cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&t->pstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->fork_next, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->ev_src, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->ev_p1, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->ev_p2[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->ev_p2[1], cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(YF_E_CUDA, "variant 4: stream set-up"));
    cudaError_t e = tb_prepare();
    if (e != cudaSuccess) return bail(cuda_fail(e, "variant 4: shared-memory opt-in"));
    return YF_OK;
}

// one time step over the whole grid (stencil only; the caller adds the epilogue)
cudaError_t tb_single(yf_grid *g, cudaStream_t s)
{
    TbPlan &t = *g->tb;
    t.chained = false;
    cudaError_t e = launch_tma_plan<float>(t.full, g->tile_y, 2 * g->cur + g->hpar, g->status, s, &g->side);
    if (e != cudaSuccess) return e;
    g->cur = (g->cur + 1) % 3;
    g->hpar ^= 1;
    return cudaSuccess;
}

// A step's epilogue on the two-step path: the source (Eq. 3) on the main stream, where the
// next step reads it; the port integrals (Eq. 4) and running transforms on the side stream,
// after the source, recording `done` there.  ev (tracing, may be null) brackets the source on
// s (q0, q0 + 1) and the side-stream kernel (q1, q1 + 1).
static cudaError_t tb_epilogue(yf_grid *g, cudaStream_t s, cudaEvent_t done, const cudaEvent_t *ev, int q0,
                               int q1)
{
    TbPlan &t = *g->tb;
    cudaError_t e;
    EpiParams<float> E = epi_params<float>(g);
    if (ev && (e = cudaEventRecord(ev[q0], s)) != cudaSuccess) return e;
    if ((e = launch_epi_source<float>(E, s)) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[q0 + 1], s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(t.ev_src, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(t.pstream, t.ev_src, 0)) != cudaSuccess) return e;
    E.skip_source = 1;
    if (ev && (e = cudaEventRecord(ev[q1], t.pstream)) != cudaSuccess) return e;
    if ((e = launch_epilogue<float>(E, t.pstream)) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[q1 + 1], t.pstream)) != cudaSuccess) return e;
    return cudaEventRecord(done, t.pstream);
}

// two time steps with both epilogues: the box n -> n+2 on a side stream, concurrently the
// frame n -> n+1 and its epilogue; then, once the box is done, the frame n+1 -> n+2 and its
// epilogue.  Buffers rotate A -> B -> C (B = A + 1, C = A + 2 mod 3), so the pair k+1 writes
// the buffer that pair k's first port epilogue reads (its box kernel waits for ev_p1) and the
// pair k+2 writes the one that pair k's second port epilogue reads (its first frame step waits
// for ev_p2 of that parity); the first two pairs after a join need no such wait.
// ev (tracing, may be null): 12 events: around the box kernel on its stream (0, 1), around
// each frame step and source on s (2..4 first step, 5..7 second), around each side-stream port
// epilogue (8, 9 and 10, 11)
cudaError_t tb_pair(yf_grid *g, cudaStream_t s, const cudaEvent_t *ev)
{
    TbPlan &t = *g->tb;
    const int r = g->cur, h = g->hpar, r1 = (r + 1) % 3;
    const int k = t.npair;
    cudaError_t e;
    const bool box = t.count > 0;
    auto mark = [&](int q, cudaStream_t st) { return ev ? cudaEventRecord(ev[q], st) : cudaSuccess; };
    if (box) {
        // a pair that follows one in the same call waits only for the previous pair's second
        // frame step, not for its epilogue: the box reads no node within four of the source
        // or port planes and writes neither of the buffers that epilogue uses
        if (!t.chained && (e = cudaEventRecord(t.fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(t.stream, t.chained ? t.fork_next : t.fork, 0)) != cudaSuccess) return e;
        if (k >= 1 && (e = cudaStreamWaitEvent(t.stream, t.ev_p1, 0)) != cudaSuccess) return e;
        if ((e = mark(0, t.stream)) != cudaSuccess) return e;
        if ((e = launch_tb2(t.items, t.count, t.args, t.maps, r, g->status, t.stream, t.ty)) != cudaSuccess)
            return e;
        if ((e = mark(1, t.stream)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(t.join, t.stream)) != cudaSuccess) return e;
    } else if (ev) {
        if ((e = mark(0, s)) != cudaSuccess || (e = mark(1, s)) != cudaSuccess) return e;
    }
    if (k >= 2 && (e = cudaStreamWaitEvent(s, t.ev_p2[k & 1], 0)) != cudaSuccess) return e;
    if ((e = mark(2, s)) != cudaSuccess) return e;
    if ((e = launch_tma_plan<float>(t.frame, g->tile_y, 2 * r + h, g->status, s, &g->side)) != cudaSuccess) return e;
    g->cur = r1;
    g->hpar = h ^ 1;
    if ((e = mark(3, s)) != cudaSuccess) return e;
    if ((e = tb_epilogue(g, s, t.ev_p1, ev, 3, 8)) != cudaSuccess) return e;
    if (box && (e = cudaStreamWaitEvent(s, t.join, 0)) != cudaSuccess) return e;
    // the second frame step writes the buffer the previous pair's first port epilogue read
    if (!box && k >= 1 && (e = cudaStreamWaitEvent(s, t.ev_p1, 0)) != cudaSuccess) return e;
    if ((e = mark(5, s)) != cudaSuccess) return e;
    if ((e = launch_tma_plan<float>(t.frame, g->tile_y, 2 * r1 + (h ^ 1), g->status, s, &g->side)) != cudaSuccess)
        return e;
    g->cur = (r + 2) % 3;
    g->hpar = h;
    if ((e = mark(6, s)) != cudaSuccess) return e;
    if (box) {
        if ((e = cudaEventRecord(t.fork_next, s)) != cudaSuccess) return e;
        t.chained = true;
    }
    if ((e = tb_epilogue(g, s, t.ev_p2[k & 1], ev, 6, 10)) != cudaSuccess) return e;
    t.npair = k + 1;
    return cudaSuccess;
}

cudaError_t tb_join(yf_grid *g, cudaStream_t s)
{
    TbPlan *t = g->tb;
    if (!t || t->npair == 0) return cudaSuccess;
    cudaError_t e = cudaStreamWaitEvent(s, t->ev_p2[(t->npair - 1) & 1], 0);
    t->npair = 0;
    return e;
}

void tb_unchain(yf_grid *g)
{
    if (g->tb) {
        g->tb->chained = false;
        g->tb->npair = 0;
    }
}

int tb_launches_pair(const yf_grid *g)
{
    return 2 * kinds_used(g->tb->frame) + (g->tb->count > 0) + 4;
}

int tb_launches_single(const yf_grid *g) { return kinds_used(g->tb->full) + 1; }

}  // namespace yf
