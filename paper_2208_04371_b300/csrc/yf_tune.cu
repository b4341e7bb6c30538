// Tile autotuner of the fused step: times every (tile_y, kseg) candidate with CUDA events on
// the grid's (or batch's) own stream, keeps the fastest, resets the solver state to zero
// (tuning happens before the first step of a solve) and caches the choice in a small JSON
// file keyed by kind, precision, size bucket (cells rounded up to a power of two) and
// whether absorbing slabs are present.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "yf_grid.h"
#include "yf_internal.h"

namespace yf {

std::string tune_key(const char *kind, yf_prec prec, long cells, int pml)
{
    int b = 0;
    while ((1L << b) < cells) ++b;
    char buf[96];
    snprintf(buf, sizeof(buf), "%s/%s/cells2^%d/%s", kind, prec == YF_FP32 ? "fp32" : "fp64", b,
             pml ? "pml" : "nopml");
    return buf;
}

static std::map<std::string, std::vector<double>> read_cache(const char *path)
{
    std::map<std::string, std::vector<double>> m;
    FILE *fp = path ? fopen(path, "r") : nullptr;
    if (!fp) return m;
    char line[512];
    while (fgets(line, sizeof(line), fp)) {
        char key[256];
        double a, b, c;
        if (sscanf(line, " \"%255[^\"]\" : [ %lf , %lf , %lf ]", key, &a, &b, &c) == 4)
            m[key] = {a, b, c};
    }
    fclose(fp);
    return m;
}

bool tune_cache_get(const char *path, const std::string &key, int *tile_y, int *kseg)
{
    auto m = read_cache(path);
    auto it = m.find(key);
    if (it == m.end()) return false;
    *tile_y = (int)it->second[0];
    *kseg = (int)it->second[1];
    return true;
}

void tune_cache_put(const char *path, const std::string &key, int tile_y, int kseg, double ms)
{
    if (!path) return;
    auto m = read_cache(path);
    m[key] = {(double)tile_y, (double)kseg, ms};
    const std::string tmp = std::string(path) + ".tmp";
    FILE *fp = fopen(tmp.c_str(), "w");
    if (!fp) return;
    fprintf(fp, "{\n");
    size_t k = 0;
    for (auto &kv : m)
        fprintf(fp, "  \"%s\": [%d, %d, %.6f]%s\n", kv.first.c_str(), (int)kv.second[0],
                (int)kv.second[1], kv.second[2], ++k < m.size() ? "," : "");
    fprintf(fp, "}\n");
    fclose(fp);
    rename(tmp.c_str(), path);
}

static const int kTiles[] = {4, 8, 16};
static const int kSegs[] = {8, 16, 32};

}  // namespace yf

using namespace yf;

extern "C" yf_status yf_autotune(yf_grid *g, const char *cache_path, int reps, int *tile_y_out,
                                 int *kseg_out)
{
    if (!g) return fail(YF_E_INVALID, "yf_autotune: NULL grid");
    if (g->steps_done != 0) return fail(YF_E_STATE, "yf_autotune must precede the first step");
    if (reps < 1) reps = 4;
    const int pml = g->pml_n > 0 && (g->bc[0] || g->bc[1] || g->bc[2] || g->bc[3] || g->bc[4] || g->bc[5]);
    const std::string key = tune_key("grid", g->prec, (long)g->nx * g->ny * g->nz, pml);
    int ty = 8, ks = 16;
    if (!tune_cache_get(cache_path, key, &ty, &ks)) {
        double best = 1e30;
        cudaEvent_t e0, e1;
        YF_CUDA_TRY(cudaEventCreate(&e0));
        YF_CUDA_TRY(cudaEventCreate(&e1));
        for (int t : kTiles)
            for (int k : kSegs) {
                yf_status st = yf_set_variant(g, 2, t, k);
                if (st == YF_OK) st = finalize(g);
                if (st != YF_OK) return st;
                cudaError_t e = step_direct(g, g->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e0, g->stream);
                for (int r = 0; r < reps && e == cudaSuccess; ++r) e = step_direct(g, g->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, g->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) return cuda_fail(e, "yf_autotune: timing");
                const double per = ms / reps;
                if (per < best) { best = per; ty = t; ks = k; }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        tune_cache_put(cache_path, key, ty, ks, best);
    }
    yf_status st = yf_set_variant(g, 2, ty, ks);
    if (st != YF_OK) return st;
    st = reset_state(g);
    if (st != YF_OK) return st;
    if (tile_y_out) *tile_y_out = ty;
    if (kseg_out) *kseg_out = ks;
    return YF_OK;
}
