// Launch tuning: how many top tree levels the traversal kernels stage in
// shared memory.  Staging saves the latency of the first loads of every query
// but takes shared memory from the same on-chip array as the L1 cache, which
// the deeper levels need; the best depth depends on the tree and the queries,
// so it is measured (kdt_autotune) and remembered per shape
// (GPU, D, k bucket, floor(log2 N)), in memory and optionally in a JSON file.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kdt_learned.cuh"
#include "kdt_query.cuh"

namespace kdt {
namespace {

constexpr int DEFAULT_STAGE_LEVELS = 0;

using ShapeKey = std::tuple<std::string, int, int, int>;  // gpu, D, k bucket, log2 N

std::mutex g_mu;
std::map<ShapeKey, int> g_tuned;

int k_bucket(int k)
{
    if (k <= 1)
        return 0;
    if (k <= 2)
        return 1;
    if (k <= 4)
        return 2;
    if (k <= 8)
        return 3;
    if (k <= 16)
        return 4;
    return 5;
}

std::string gpu_name()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess)
        return "unknown";
    std::string n = p.name;
    for (char &c : n)
        if (c == '"' || c == '\\')
            c = '_';
    return n;
}

ShapeKey shape_of(const kdt_tree *t, int k)
{
    return ShapeKey(gpu_name(), t->D, k_bucket(k), floor_log2((uint64_t)t->N));
}

}  // namespace

int stage_levels_for(const kdt_tree *t, int k)
{
    if (t->stage_levels >= 0)
        return t->stage_levels;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_tuned.empty()) {
        auto it = g_tuned.find(shape_of(t, k));
        if (it != g_tuned.end())
            return it->second;
    }
    return DEFAULT_STAGE_LEVELS;
}

}  // namespace kdt

using namespace kdt;

extern "C" {

int kdt_set_stage_levels(kdt_tree *t, int levels)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (levels < -1 || levels > 16)
        return set_error(KDT_EINVAL, "levels must be in [-1, 16] (got %d)", levels);
    const int per = t->layout == 2 ? 32 : 16;
    if (levels > 0 && (((int64_t)1 << levels) - 1) * per > 160 * 1024)
        return set_error(KDT_EINVAL, "%d staged levels exceed the shared-memory budget", levels);
    t->stage_levels = levels;
    return KDT_OK;
}

int kdt_autotune(kdt_tree *t, const float *d_q, int64_t Q, int k, int flags, int *best_levels, float *best_ms,
                 void *stream)
{
    if (!t || !d_q || Q < 1 || k < 1 || k > 64)
        return set_error(KDT_EINVAL, "bad autotune arguments");
    if (flags & KDT_LEARNED)
        return set_error(KDT_EINVAL, "autotune the plain traversal (no KDT_LEARNED)");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = Q < ((int64_t)1 << 20) ? Q : ((int64_t)1 << 20);
    int32_t *ids = nullptr;
    float *d2 = nullptr;
    KDT_CUDA(cudaMallocAsync(&ids, (size_t)n * k * 4, s));
    KDT_CUDA(cudaMallocAsync(&d2, (size_t)n * k * 4, s));
    cudaEvent_t e0, e1;
    KDT_CUDA(cudaEventCreate(&e0));
    KDT_CUDA(cudaEventCreate(&e1));
    const int saved = t->stage_levels;
    const int per = t->layout == 2 ? 32 : 16;
    const int cand[] = {0, 4, 6, 8, 10, 11, 12};
    int best = DEFAULT_STAGE_LEVELS;
    float best_t = 3.4e38f;
    int rc = KDT_OK;
    for (int c : cand) {
        if (c > 0 && (((int64_t)1 << c) - 1) * per > 64 * 1024)
            continue;
        t->stage_levels = c;
        float ms = 0.f;
        for (int rep = 0; rep < 3 && rc == KDT_OK; ++rep) {
            rc = run_query(t, d_q, n, k, INFINITY, flags & ~KDT_NO_STAGE, MODE_RESULTS, ids, d2, nullptr, s);
            if (rc == KDT_OK && rep == 0)
                rc = cudaEventRecord(e0, s) == cudaSuccess ? KDT_OK : set_error(KDT_ECUDA, "event record");
        }
        if (rc != KDT_OK)
            break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = set_error(KDT_ECUDA, "event timing failed");
            break;
        }
        ms *= 0.5f;  // two timed launches
        if (ms < best_t) {
            best_t = ms;
            best = c;
        }
    }
    t->stage_levels = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(ids, s);
    cudaFreeAsync(d2, s);
    if (rc != KDT_OK)
        return rc;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_tuned[shape_of(t, k)] = best;
    }
    if (best_levels)
        *best_levels = best;
    if (best_ms)
        *best_ms = best_t;
    return KDT_OK;
}

int kdt_tuning_save(const char *path)
{
    if (!path)
        return set_error(KDT_EINVAL, "path is NULL");
    std::vector<std::pair<ShapeKey, int>> rows;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        rows.assign(g_tuned.begin(), g_tuned.end());
    }
    FILE *f = fopen(path, "w");
    if (!f)
        return set_error(KDT_EIO, "cannot open %s for writing", path);
    bool ok = fprintf(f, "[\n") > 0;
    for (size_t i = 0; i < rows.size() && ok; ++i) {
        const ShapeKey &key = rows[i].first;
        ok = fprintf(f, "  {\"gpu\": \"%s\", \"D\": %d, \"k_bucket\": %d, \"log2n\": %d, \"stage_levels\": %d}%s\n",
                     std::get<0>(key).c_str(), std::get<1>(key), std::get<2>(key), std::get<3>(key), rows[i].second,
                     i + 1 < rows.size() ? "," : "") > 0;
    }
    ok = ok && fprintf(f, "]\n") > 0;
    ok = (fclose(f) == 0) && ok;
    return ok ? KDT_OK : set_error(KDT_EIO, "write to %s failed", path);
}

// reads the format kdt_tuning_save writes (one object per line)
int kdt_tuning_load(const char *path)
{
    if (!path)
        return set_error(KDT_EINVAL, "path is NULL");
    FILE *f = fopen(path, "r");
    if (!f)
        return set_error(KDT_EIO, "cannot open %s", path);
    char line[512];
    std::vector<std::pair<ShapeKey, int>> rows;
    bool bad = false;
    while (fgets(line, sizeof line, f)) {
        const char *g = strstr(line, "\"gpu\": \"");
        if (!g)
            continue;
        g += 8;
        const char *ge = strchr(g, '"');
        int D, kb, l2, lv;
        if (!ge || sscanf(ge, "\", \"D\": %d, \"k_bucket\": %d, \"log2n\": %d, \"stage_levels\": %d", &D, &kb, &l2,
                          &lv) != 4 || lv < 0 || lv > 16) {
            bad = true;
            break;
        }
        rows.emplace_back(ShapeKey(std::string(g, ge - g), D, kb, l2), lv);
    }
    fclose(f);
    if (bad)
        return set_error(KDT_EIO, "%s is not a tuning file", path);
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto &r : rows)
        g_tuned[r.first] = r.second;
    return KDT_OK;
}

}  // extern "C"
