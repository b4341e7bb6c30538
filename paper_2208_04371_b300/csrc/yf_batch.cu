// Batched solve of many independent line instances (uneven sizes) sharing one time step.
//
// Each instance is an ordinary yf_grid configured through the single-grid set-up calls
// (materials, sheets, boundaries, CPML, source, ports), so every instance computes exactly
// what the single-grid path computes.  A batch step is at most six launches for all
// instances together: the CPML-free interior work items, up to four kinds of CPML frame work
// items (x, y, z, or all slabs; each on its own side stream), and a one-block-per-instance
// port epilogue.  A work item is one 32 x tile_y node column of one instance over a
// z-segment; per-instance kernel arguments and tensor maps live in device memory, two sets
// each (field-buffer parity 0 and 1).  Chunks of steps replay from captured CUDA graphs.
//
// With variant 4 (FP32), every instance with an inner box (the single-grid variant-4 box) has
// it advanced two steps per pass: a pair of steps is one box-kernel launch over every
// instance's box items, beside the one-step frame kinds of the first step and their epilogue,
// then the frame kinds of the second step and theirs.  Instances then keep three field
// buffers; arguments and maps come in six one-step sets (2 * source buffer + H-copy parity),
// three two-step sets and three epilogue sets per instance.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "yf_grid.h"
#include "yf_internal.h"

struct yf_batch {
    std::vector<yf_grid *> g;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    yf_prec prec = YF_FP32;
    double dt = 0;
    int tile_y = 8, kseg = 16, chunk = 32;
    bool started = false;
    int cur = 0;
    long steps_done = 0;
    long cells = 0;
    yf::TmaPlan plan = {};            // work items, arguments, tensor maps of all instances
    void *eps = nullptr;              // EpiParams<T>[2 n]
    int *status = nullptr;            // stencil error bits of the batch
    yf::SideStream side = {};
    cudaGraphExec_t graph[2] = {};
    // variant 4 (FP32): two time steps per pass over each instance's inner box.  Every instance
    // keeps three field buffers; all rotate together (cur in 0..2, hpar the H-copy parity)
    int variant = 2;
    int hpar = 0;
    yf::TmaPlan full4 = {}, frame4 = {};   // one-step items (6 argument sets per instance); frame4 shares args and maps
    yf::BatchItem *box_items = nullptr;    // two-step items of every instance's box
    int box_count = 0;
    yf::TbArgs *tb_args = nullptr;         // [n][3] by source buffer
    CUtensorMap *tb_maps = nullptr;        // [n][3][3]
    void *eps3 = nullptr;                  // EpiParams<float>[n][3], by current buffer
    cudaStream_t bstream = nullptr;        // the box kernel's stream
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraphExec_t graph4[6] = {};        // chunks by state 2 cur + hpar
};

namespace yf {

template <typename T>
yf_status build_plan(const std::vector<yf_grid *> &grids, int tile_y, int kseg, TmaPlan *pl)
{
    const int n = (int)grids.size();
    std::vector<BatchItem> items[5];
    std::vector<FusedArgs<T>> args(2 * n);
    std::vector<CUtensorMap> maps(4 * n);
    for (int q = 0; q < n; ++q) {
        yf_grid *g = grids[q];
        tma_items(q, g->nx, g->ny, g->nz, kseg, tile_y, g->pml_n, g->pml_lo, g->pml_hi, items);
        const int c0 = g->cur, h0 = g->hpar;
        for (int par = 0; par < 2; ++par) {
            g->cur = par;
            g->hpar = par;
            args[2 * q + par] = fused_args<T>(g);
            maps[2 * (2 * q + par) + 0] = g->tmF[par];
            maps[2 * (2 * q + par) + 1] = g->tmC;
        }
        g->cur = c0;
        g->hpar = h0;
    }
    std::vector<BatchItem> all;
    for (int k = 0; k < 5; ++k) {
        pl->offset[k] = (int)all.size();
        pl->count[k] = (int)items[k].size();
        all.insert(all.end(), items[k].begin(), items[k].end());
    }
    YF_CUDA_TRY(cudaMalloc(&pl->items, std::max<size_t>(1, all.size()) * sizeof(BatchItem)));
    YF_CUDA_TRY(cudaMemcpy(pl->items, all.data(), all.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    YF_CUDA_TRY(cudaMalloc(&pl->args, args.size() * sizeof(FusedArgs<T>)));
    YF_CUDA_TRY(cudaMemcpy(pl->args, args.data(), args.size() * sizeof(FusedArgs<T>), cudaMemcpyHostToDevice));
    YF_CUDA_TRY(cudaMalloc(&pl->maps, maps.size() * sizeof(CUtensorMap)));
    YF_CUDA_TRY(cudaMemcpy(pl->maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    return YF_OK;
}

template yf_status build_plan<float>(const std::vector<yf_grid *> &, int, int, TmaPlan *);
template yf_status build_plan<double>(const std::vector<yf_grid *> &, int, int, TmaPlan *);

void free_plan(TmaPlan *pl)
{
    cudaFree(pl->items);
    cudaFree(pl->args);
    cudaFree(pl->maps);
    *pl = TmaPlan{};
}

namespace {

void free_device(yf_batch *b)
{
    free_plan(&b->plan);
    cudaFree(b->eps); b->eps = nullptr;
    for (int p = 0; p < 2; ++p)
        if (b->graph[p]) { cudaGraphExecDestroy(b->graph[p]); b->graph[p] = nullptr; }
    cudaFree(b->frame4.items);
    b->frame4 = TmaPlan{};
    free_plan(&b->full4);
    cudaFree(b->box_items); b->box_items = nullptr;
    b->box_count = 0;
    cudaFree(b->tb_args); b->tb_args = nullptr;
    cudaFree(b->tb_maps); b->tb_maps = nullptr;
    cudaFree(b->eps3); b->eps3 = nullptr;
    for (int p = 0; p < 6; ++p)
        if (b->graph4[p]) { cudaGraphExecDestroy(b->graph4[p]); b->graph4[p] = nullptr; }
}

template <typename X>
yf_status upload(X **dst, const std::vector<X> &v)
{
    YF_CUDA_TRY(cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(X)));
    if (!v.empty()) YF_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice));
    return YF_OK;
}

yf_status upload_kinds(const std::vector<BatchItem> items[5], TmaPlan *pl)
{
    std::vector<BatchItem> all;
    for (int k = 0; k < 5; ++k) {
        pl->offset[k] = (int)all.size();
        pl->count[k] = (int)items[k].size();
        all.insert(all.end(), items[k].begin(), items[k].end());
    }
    return upload(&pl->items, all);
}

// every instance follows the batch's buffer rotation (readbacks use each grid's own state)
void set_state(yf_batch *b, int cur, int hpar)
{
    b->cur = cur;
    b->hpar = hpar;
    for (yf_grid *g : b->g) {
        g->cur = cur;
        g->hpar = hpar;
    }
}

// Variant 4 tables: per instance a third field buffer (equal to the current one: nodes no kernel
// writes must agree in all three), maps for it, its box (one two-step segment per tile column),
// its one-step and two-step arguments and its epilogue parameters by buffer.
yf_status prepare4(yf_batch *b)
{
    const int n = (int)b->g.size();
    std::vector<BatchItem> full[5], frame[5], two;
    std::vector<FusedArgs<float>> fa(6 * (size_t)n);
    std::vector<CUtensorMap> fm(12 * (size_t)n), tm(9 * (size_t)n);
    std::vector<TbArgs> ta(3 * (size_t)n);
    std::vector<EpiParams<float>> eps(3 * (size_t)n);
    for (int q = 0; q < n; ++q) {
        yf_grid *g = b->g[q];
        if (6 * g->npts > 2147483647L)
            return fail(YF_E_INVALID, "instance %d: variant 4 needs 6 (nz+1)(ny+1) px < 2^31", q);
        if (!g->buf[2]) {
            const size_t bytes = 6 * g->npts * g->esz;
            YF_CUDA_TRY(cudaMalloc(&g->buf[2], bytes));
            for (int r = 0; r < 3; ++r)
                if (r != g->cur) YF_CUDA_TRY(cudaMemcpyAsync(g->buf[r], g->buf[g->cur], bytes, cudaMemcpyDeviceToDevice, b->stream));
            g->tmap_tile_y = 0;
        }
        g->tile_y = b->tile_y;
        g->kseg = b->kseg;
        yf_status st = encode_maps(g);
        if (st != YF_OK) return st;
        int box[6] = {0, 0, 0, 0, 0, 0};
        const bool have = choose_box(g, box);
        tb_items(g, q, have, box, 8, g->nz + 1, full, frame, two, 0);
        tb_step_args(g, &fa[6 * (size_t)q], &fm[12 * (size_t)q]);
        if (have && (st = tb_box_args(g, box, 8, &ta[3 * (size_t)q], &tm[9 * (size_t)q])) != YF_OK) return st;
        const int c0 = g->cur;
        for (int r = 0; r < 3; ++r) {
            g->cur = r;
            eps[3 * (size_t)q + r] = epi_params<float>(g);
        }
        g->cur = c0;
    }
    yf_status st;
    if ((st = upload_kinds(full, &b->full4)) != YF_OK) return st;
    if ((st = upload_kinds(frame, &b->frame4)) != YF_OK) return st;
    FusedArgs<float> *fad = nullptr;
    if ((st = upload(&fad, fa)) != YF_OK) return st;
    b->full4.args = b->frame4.args = fad;
    if ((st = upload(&b->full4.maps, fm)) != YF_OK) return st;
    b->frame4.maps = b->full4.maps;
    b->full4.stride = b->frame4.stride = 6;
    if ((st = upload(&b->box_items, two)) != YF_OK) return st;
    b->box_count = (int)two.size();
    if ((st = upload(&b->tb_args, ta)) != YF_OK) return st;
    if ((st = upload(&b->tb_maps, tm)) != YF_OK) return st;
    EpiParams<float> *ed = nullptr;
    if ((st = upload(&ed, eps)) != YF_OK) return st;
    b->eps3 = ed;
    if (!b->bstream) YF_CUDA_TRY(cudaStreamCreateWithFlags(&b->bstream, cudaStreamNonBlocking));
    if (!b->fork) YF_CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    if (!b->join) YF_CUDA_TRY(cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming));
    YF_CUDA_TRY(tb_prepare());
    set_state(b, b->g.empty() ? 0 : b->g[0]->cur, b->g.empty() ? 0 : b->g[0]->hpar);
    return YF_OK;
}

template <typename T>
yf_status build_tables(yf_batch *b)
{
    const int n = (int)b->g.size();
    yf_status st = build_plan<T>(b->g, b->tile_y, b->kseg, &b->plan);
    if (st != YF_OK) return st;
    std::vector<EpiParams<T>> eps(2 * n);
    for (int q = 0; q < n; ++q) {
        yf_grid *g = b->g[q];
        const int c0 = g->cur, h0 = g->hpar;
        for (int par = 0; par < 2; ++par) {
            g->cur = par;
            g->hpar = par;
            eps[2 * q + par] = epi_params<T>(g);
        }
        g->cur = c0;
        g->hpar = h0;
    }
    YF_CUDA_TRY(cudaMalloc(&b->eps, eps.size() * sizeof(EpiParams<T>)));
    YF_CUDA_TRY(cudaMemcpy(b->eps, eps.data(), eps.size() * sizeof(EpiParams<T>), cudaMemcpyHostToDevice));
    return YF_OK;
}

yf_status prepare(yf_batch *b)
{
    if (b->started) return YF_OK;
    for (yf_grid *g : b->g) {
        yf_status st = finalize(g);
        if (st != YF_OK) return st;
        g->tile_y = b->tile_y;
        g->kseg = b->kseg;
        st = encode_maps(g);
        if (st != YF_OK) return st;
    }
    yf_status st = b->variant == 4 ? prepare4(b) : b->prec == YF_FP32 ? build_tables<float>(b) : build_tables<double>(b);
    if (st != YF_OK) return st;
    YF_CUDA_TRY(side_create(&b->side));
    b->started = true;
    return YF_OK;
}

// variant 4: one step over every instance (all items), then the epilogue at the new buffer
cudaError_t single4(yf_batch *b)
{
    const int r = b->cur, h = b->hpar, r1 = (r + 1) % 3;
    cudaError_t e = launch_tma_plan<float>(b->full4, b->tile_y, 2 * r + h, b->status, b->stream, &b->side);
    if (e != cudaSuccess) return e;
    set_state(b, r1, h ^ 1);
    return launch_epilogue_batch<float>((const EpiParams<float> *)b->eps3, (int)b->g.size(), r1, b->stream, 3);
}

// variant 4: two steps.  The boxes n -> n+2 on the box stream, beside the frames n -> n+1 and
// their epilogue; once the boxes are done (their outer node layer at n+1 is in the middle
// buffer) the frames n+1 -> n+2 and their epilogue.  The epilogues touch only source and port
// planes, which no box reads or writes.  A pair's box kernel waits for everything queued
// before it on the batch stream.
cudaError_t pair4(yf_batch *b)
{
    const int n = (int)b->g.size();
    const int r = b->cur, h = b->hpar, r1 = (r + 1) % 3, r2 = (r + 2) % 3;
    const EpiParams<float> *E = (const EpiParams<float> *)b->eps3;
    const bool box = b->box_count > 0;
    cudaError_t e;
    if (box) {
        if ((e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(b->bstream, b->fork, 0)) != cudaSuccess) return e;
        if ((e = launch_tb2(b->box_items, b->box_count, b->tb_args, b->tb_maps, r, b->status, b->bstream, 8)) !=
            cudaSuccess)
            return e;
        if ((e = cudaEventRecord(b->join, b->bstream)) != cudaSuccess) return e;
    }
    if ((e = launch_tma_plan<float>(b->frame4, b->tile_y, 2 * r + h, b->status, b->stream, &b->side)) != cudaSuccess)
        return e;
    if ((e = launch_epilogue_batch<float>(E, n, r1, b->stream, 3)) != cudaSuccess) return e;
    if (box && (e = cudaStreamWaitEvent(b->stream, b->join, 0)) != cudaSuccess) return e;
    if ((e = launch_tma_plan<float>(b->frame4, b->tile_y, 2 * r1 + (h ^ 1), b->status, b->stream, &b->side)) !=
        cudaSuccess)
        return e;
    if ((e = launch_epilogue_batch<float>(E, n, r2, b->stream, 3)) != cudaSuccess) return e;
    set_state(b, r2, h);
    return cudaSuccess;
}

template <typename T>
cudaError_t step_t(yf_batch *b)
{
    const int n = (int)b->g.size();
    cudaError_t e = launch_tma_plan<T>(b->plan, b->tile_y, b->cur, b->status, b->stream, &b->side);
    if (e != cudaSuccess) return e;
    b->cur ^= 1;
    for (yf_grid *g : b->g) {
        g->cur ^= 1;
        g->hpar ^= 1;
    }
    return launch_epilogue_batch<T>((const EpiParams<T> *)b->eps, n, b->cur, b->stream);
}

cudaError_t step_once(yf_batch *b)
{
    if (b->variant == 4) return single4(b);
    return b->prec == YF_FP32 ? step_t<float>(b) : step_t<double>(b);
}

// variant 4: a chunk of pairs from state (cur, hpar); the state is restored after the capture
// and advanced by the caller after each replay
yf_status capture4(yf_batch *b)
{
    cudaGraph_t graph = nullptr;
    const int c0 = b->cur, h0 = b->hpar, key = 2 * c0 + h0;
    YF_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int t = 0; t + 1 < b->chunk && e == cudaSuccess; t += 2) e = pair4(b);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    set_state(b, c0, h0);
    if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "capturing batch chunk"); }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph4[key], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { b->graph4[key] = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    return YF_OK;
}

yf_status capture(yf_batch *b)
{
    cudaGraph_t graph = nullptr;
    const int c0 = b->cur;
    YF_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < b->chunk && e == cudaSuccess; ++t) e = step_once(b);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "capturing batch chunk"); }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph[c0], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { b->graph[c0] = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    return YF_OK;
}

}  // namespace
}  // namespace yf

using namespace yf;

extern "C" {

yf_status yf_batch_create(int n, const yf_instance_desc *d, double dt, yf_prec prec, void *stream,
                          yf_batch **out)
{
    if (!out || !d || n < 1) return fail(YF_E_INVALID, "yf_batch_create: need n >= 1 descriptors");
    *out = nullptr;
    double lim = 0.0;
    for (int q = 0; q < n; ++q) {
        const double l = courant_limit_dt(d[q].dx, d[q].dy, d[q].dz);
        lim = q == 0 ? l : std::min(lim, l);
    }
    if (dt <= 0) dt = 0.99 * lim;
    if (dt > lim * (1.0 + 1e-12))
        return fail(YF_E_UNSTABLE, "dt = %.6g s exceeds the Courant limit %.6g s of an instance", dt, lim);
    yf_batch *b = new (std::nothrow) yf_batch();
    if (!b) return fail(YF_E_OOM, "yf_batch_create: host allocation failed");
    b->prec = prec;
    b->dt = dt;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaStreamCreate"); }
        b->own_stream = true;
    }
    yf_status st = YF_OK;
    if (cudaMalloc(&b->status, sizeof(int)) != cudaSuccess || cudaMemset(b->status, 0, sizeof(int)) != cudaSuccess)
        st = fail(YF_E_OOM, "yf_batch_create: status word");
    for (int q = 0; q < n && st == YF_OK; ++q) {
        const yf_instance_desc &D = d[q];
        yf_grid *g = nullptr;
        st = yf_grid_create(D.nx, D.ny, D.nz, D.dx, D.dy, D.dz, dt, prec, b->stream, &g);
        if (st != YF_OK) break;
        b->g.push_back(g);
        g->variant = 1;   // stepping is done by the batch; no per-grid side stream
        b->cells += (long)D.nx * D.ny * D.nz;
        if (D.ids) st = yf_set_materials(g, D.ids, YF_HOST, D.nmat, D.eps_r, D.sigma, D.mu_r, D.is_pec);
        for (int s = 0; s < D.nsheets && st == YF_OK; ++s) {
            const int *sh = D.sheets + 6 * s;
            st = yf_add_pec_sheet(g, sh[0], sh[1], sh[2], sh[3], sh[4], sh[5]);
        }
        if (st == YF_OK) st = yf_set_boundaries(g, D.bc);
        if (st == YF_OK)
            st = yf_set_pml(g, D.pml_cells, D.pml_order, D.pml_sigma_scale, D.pml_kappa_max, D.pml_alpha_max);
        if (st == YF_OK && D.src.kind != YF_WAVE_NONE)
            st = yf_set_source(g, 0, D.src_plane, D.src_j0, D.src_j1, D.src_k0, D.src_k1, &D.src);
        for (int p = 0; p < D.nports && st == YF_OK; ++p)
            st = yf_add_port(g, &D.ports[p], D.nfreq, D.freqs, nullptr);
        if (st != YF_OK) {
            char msg[600];
            snprintf(msg, sizeof(msg), "instance %d: %s", q, yf_last_error());
            st = fail(st, "%s", msg);
        }
    }
    if (st != YF_OK) {
        yf_batch_destroy(b);
        return st;
    }
    *out = b;
    return YF_OK;
}

yf_status yf_batch_destroy(yf_batch *b)
{
    if (!b) return YF_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_device(b);
    for (yf_grid *g : b->g) yf_grid_destroy(g);
    cudaFree(b->status);
    side_destroy(&b->side);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->bstream) cudaStreamDestroy(b->bstream);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return YF_OK;
}

yf_status yf_batch_set_tiling(yf_batch *b, int tile_y, int kseg)
{
    if (!b) return fail(YF_E_INVALID, "yf_batch_set_tiling: NULL batch");
    if (tile_y != 4 && tile_y != 8 && tile_y != 16) return fail(YF_E_INVALID, "tile_y must be 4, 8 or 16");
    if (kseg < 1 || kseg > kMaxKseg) return fail(YF_E_INVALID, "kseg must be 1..%d", kMaxKseg);
    YF_CUDA_TRY(cudaStreamSynchronize(b->stream));
    free_device(b);
    b->tile_y = tile_y;
    b->kseg = kseg;
    b->started = false;   // items, tables and maps are rebuilt at the next step
    return YF_OK;
}

yf_status yf_batch_set_variant(yf_batch *b, int variant)
{
    if (!b) return fail(YF_E_INVALID, "yf_batch_set_variant: NULL batch");
    if (variant == b->variant) return YF_OK;
    if (variant != 4) return fail(YF_E_INVALID, "yf_batch_set_variant: variant must be 4 (the default is 2)");
    if (b->prec != YF_FP32) return fail(YF_E_INVALID, "variant 4 needs FP32 fields");
    if (b->steps_done != 0) return fail(YF_E_STATE, "yf_batch_set_variant must precede the first step");
    if (b->chunk % 2) return fail(YF_E_STATE, "variant 4 needs an even chunk");
    YF_CUDA_TRY(cudaStreamSynchronize(b->stream));
    free_device(b);
    b->variant = 4;
    b->started = false;   // tables, third buffers and maps are built at the next step
    return YF_OK;
}

yf_status yf_batch_step(yf_batch *b, long n)
{
    if (!b || n < 0) return fail(YF_E_INVALID, "yf_batch_step: bad argument");
    yf_status st = prepare(b);
    if (st != YF_OK) return st;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    YF_CUDA_TRY(cudaStreamIsCapturing(b->stream, &cs));
    long done = 0;
    if (b->variant == 4) {
        if (cs == cudaStreamCaptureStatusNone && n >= b->chunk)
            for (; done + b->chunk <= n; done += b->chunk) {
                const int key = 2 * b->cur + b->hpar;
                if (!b->graph4[key] && (st = capture4(b)) != YF_OK) return st;
                YF_CUDA_TRY(cudaGraphLaunch(b->graph4[key], b->stream));
                // an even chunk of pairs: the buffers rotate by chunk mod 3, the H copy stays
                set_state(b, (b->cur + b->chunk) % 3, b->hpar);
            }
        for (; done + 2 <= n; done += 2) YF_CUDA_TRY(pair4(b));
        if (done < n) {
            YF_CUDA_TRY(single4(b));
            ++done;
        }
        b->steps_done += n;
        for (yf_grid *g : b->g) g->steps_done += n;
        return YF_OK;
    }
    if (cs == cudaStreamCaptureStatusNone && n >= b->chunk) {
        if (!b->graph[b->cur]) {
            st = capture(b);
            if (st != YF_OK) return st;
        }
        for (; done + b->chunk <= n; done += b->chunk) {
            YF_CUDA_TRY(cudaGraphLaunch(b->graph[b->cur], b->stream));
            // a chunk is even: the buffer parity is unchanged after the replay
        }
    }
    for (; done < n; ++done) YF_CUDA_TRY(step_once(b));
    b->steps_done += n;
    for (yf_grid *g : b->g) g->steps_done += n;
    return YF_OK;
}

yf_status yf_batch_sync(yf_batch *b)
{
    if (!b) return fail(YF_E_INVALID, "yf_batch_sync: NULL batch");
    YF_CUDA_TRY(cudaStreamSynchronize(b->stream));
    int st = 0;
    YF_CUDA_TRY(cudaMemcpy(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & 4) return fail(YF_E_CUDA, "batched step: shared memory base not 128-byte aligned");
    if (st & 2) return fail(YF_E_TIMEOUT, "a bounded device wait of the batched step gave up");
    for (size_t q = 0; q < b->g.size(); ++q) {
        yf_status s = yf_sync(b->g[q]);
        if (s != YF_OK) return fail(s, "instance %zu: %s", q, yf_last_error());
    }
    return YF_OK;
}

yf_status yf_batch_grid(yf_batch *b, int inst, yf_grid **g)
{
    if (!b || !g || inst < 0 || inst >= (int)b->g.size()) return fail(YF_E_INVALID, "yf_batch_grid: bad instance");
    *g = b->g[inst];
    return YF_OK;
}

yf_status yf_batch_info(yf_batch *b, int *n, long *cells, double *dt, long *steps)
{
    if (!b) return fail(YF_E_INVALID, "yf_batch_info: NULL batch");
    if (n) *n = (int)b->g.size();
    if (cells) *cells = b->cells;
    if (dt) *dt = b->dt;
    if (steps) *steps = b->steps_done;
    return YF_OK;
}

yf_status yf_batch_autotune(yf_batch *b, const char *cache_path, int reps, int *tile_y_out,
                            int *kseg_out)
{
    if (!b) return fail(YF_E_INVALID, "yf_batch_autotune: NULL batch");
    if (b->steps_done != 0) return fail(YF_E_STATE, "yf_batch_autotune must precede the first step");
    if (reps < 1) reps = 3;
    int pml = 0;
    for (yf_grid *g : b->g) pml |= g->pml_n > 0;
    const std::string key = tune_key("batch", b->prec, b->cells, pml);
    int ty = 8, ks = 16;
    if (!tune_cache_get(cache_path, key, &ty, &ks)) {
        static const int tiles[] = {4, 8, 16}, segs[] = {8, 16, 32};
        double best = 1e30;
        cudaEvent_t e0, e1;
        YF_CUDA_TRY(cudaEventCreate(&e0));
        YF_CUDA_TRY(cudaEventCreate(&e1));
        for (int t : tiles)
            for (int k : segs) {
                yf_status st = yf_batch_set_tiling(b, t, k);
                if (st == YF_OK) st = prepare(b);
                if (st != YF_OK) return st;
                cudaError_t e = step_once(b);
                if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
                for (int r = 0; r < reps && e == cudaSuccess; ++r) e = step_once(b);
                if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) return cuda_fail(e, "yf_batch_autotune: timing");
                const double per = ms / reps;
                if (per < best) { best = per; ty = t; ks = k; }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        tune_cache_put(cache_path, key, ty, ks, best);
    }
    yf_status st = yf_batch_set_tiling(b, ty, ks);
    for (size_t q = 0; q < b->g.size() && st == YF_OK; ++q) st = reset_state(b->g[q]);
    if (st != YF_OK) return st;
    if (tile_y_out) *tile_y_out = ty;
    if (kseg_out) *kseg_out = ks;
    return YF_OK;
}

yf_status yf_batch_read_port_dft(yf_batch *b, int inst, int port, int kind, double *V_re,
                                 double *V_im, double *I_re, double *I_im)
{
    if (!b || inst < 0 || inst >= (int)b->g.size()) return fail(YF_E_INVALID, "yf_batch_read_port_dft: bad instance");
    return yf_read_port_dft(b->g[inst], port, kind, V_re, V_im, I_re, I_im);
}

}  // extern "C"
