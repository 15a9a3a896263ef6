// Launch tuning of the traversal kernels.  Three choices never change a result
// (every combination processes the same nodes in the same order) but move its
// speed, and the best values depend on how much work a query does:
//   * stage_levels: top tree levels staged in shared memory (saves the latency
//     of the first loads, but the shared memory comes out of the same on-chip
//     array as the L1 cache that the deeper levels need);
//   * claim_steps: traversal steps a lane takes between two claim rounds of its
//     warp (long runs amortise the warp vote; a lane whose query has ended
//     waits for the round);
//   * inline_depth: depth of the bottom subtrees one step processes whole
//     (2 or 3 save steps on long queries; 1 avoids the extra up-front loads
//     that short queries rarely use; 0 selects the simplest kernel, one node
//     per step, where it applies: ordered, k <= 16, D <= 4, no staging);
//   * light_run: steps a lane takes per call while they are light, so that
//     the heavy steps (whole bottom subtrees) of a warp's lanes coincide
//     (1 for long queries; 4 or 8 pay for short ones);
//   * large_k_list (k > 16): the k-best heap in shared memory (pays for short
//     queries) or in global scratch (full occupancy and L1; pays for long
//     ones), chosen by the sample's processed nodes per query.
// kdt_autotune measures them on the caller's queries and remembers the best
// per shape (GPU, D, k bucket, floor(log2 N)), in memory and optionally in a
// JSON file; without a tuning the defaults below apply.
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
constexpr int DEFAULT_INLINE_DEPTH = 2;
constexpr int DEFAULT_LIGHT_RUN = 1;
constexpr int DEFAULT_LARGE_K_LIST = KDT_LIST_SHARED;
// measured on GB300: 64 steps per claim round is best for k >= 2 on every
// workload tried, 32 for fcp
int default_claim_steps(int k) { return k <= 1 ? 32 : 64; }

struct Tuned {
    int stage_levels;
    int claim_steps;
    int inline_depth;
    int light_run;
    int large_k_list;
};

using ShapeKey = std::tuple<std::string, int, int, int>;  // gpu, D, k bucket, log2 N

std::mutex g_mu;
std::map<ShapeKey, Tuned> g_tuned;

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

bool tuned_for(const kdt_tree *t, int k, Tuned *out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_tuned.empty())
        return false;
    auto it = g_tuned.find(shape_of(t, k));
    if (it == g_tuned.end())
        return false;
    *out = it->second;
    return true;
}

bool stage_fits(const kdt_tree *t, int levels, int budget)
{
    const int per = t->layout == 2 ? 32 : 16;
    return levels <= 0 || (((int64_t)1 << levels) - 1) * per <= budget;
}

}  // namespace

int default_claim_steps_k(int k) { return default_claim_steps(k); }

int stage_levels_for(const kdt_tree *t, int k)
{
    if (t->stage_levels >= 0)
        return t->stage_levels;
    Tuned v;
    return tuned_for(t, k, &v) ? v.stage_levels : DEFAULT_STAGE_LEVELS;
}

int claim_steps_for(const kdt_tree *t, int k)
{
    if (t->claim_steps > 0)
        return t->claim_steps;
    Tuned v;
    return tuned_for(t, k, &v) ? v.claim_steps : default_claim_steps(k);
}

int light_run_for(const kdt_tree *t, int k)
{
    if (t->light_run > 0)
        return t->light_run;
    Tuned v;
    return tuned_for(t, k, &v) ? v.light_run : DEFAULT_LIGHT_RUN;
}

static int large_k_list_of(const kdt_tree *t, int k)
{
    if (t->large_k_list >= 0)
        return t->large_k_list;
    Tuned v;
    return tuned_for(t, k, &v) ? v.large_k_list : DEFAULT_LARGE_K_LIST;
}

bool heap_in_global(const kdt_tree *t, int k) { return k > 16 && large_k_list_of(t, k) == KDT_LIST_GLOBAL; }

int list_group_for(const kdt_tree *t, int k)
{
    if (k <= 16)
        return 1;
    const int p = large_k_list_of(t, k);
    return p == KDT_LIST_GROUP8 ? 8 : (p == KDT_LIST_GROUP4 ? 4 : 1);
}

int inline_depth_for(const kdt_tree *t, int k)
{
    if (t->inline_depth >= 0)
        return t->inline_depth;
    Tuned v;
    return tuned_for(t, k, &v) ? v.inline_depth : DEFAULT_INLINE_DEPTH;
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
    if (!stage_fits(t, levels, 160 * 1024))
        return set_error(KDT_EINVAL, "%d staged levels exceed the shared-memory budget", levels);
    t->stage_levels = levels;
    return KDT_OK;
}

int kdt_set_claim_steps(kdt_tree *t, int steps)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (steps < -1 || steps == 0 || steps > 256)
        return set_error(KDT_EINVAL, "steps must be -1 or in [1, 256] (got %d)", steps);
    t->claim_steps = steps;
    return KDT_OK;
}

int kdt_set_inline_depth(kdt_tree *t, int depth)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (depth < -1 || depth > 4)
        return set_error(KDT_EINVAL, "depth must be in [-1, 4] (got %d)", depth);
    t->inline_depth = depth;
    return KDT_OK;
}

int kdt_set_light_run(kdt_tree *t, int steps)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (steps < -1 || steps == 0 || steps > 64)
        return set_error(KDT_EINVAL, "steps must be -1 or in [1, 64] (got %d)", steps);
    t->light_run = steps;
    return KDT_OK;
}

int kdt_set_large_k_list(kdt_tree *t, int placement)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (placement < -1 || placement > KDT_LIST_GROUP8)
        return set_error(KDT_EINVAL, "placement must be -1 or one of KDT_LIST_* (got %d)", placement);
    t->large_k_list = placement;
    return KDT_OK;
}

int kdt_large_k_list(const kdt_tree *t, int k, int *placement)
{
    if (!t || k < 1 || k > 64 || !placement)
        return set_error(KDT_EINVAL, "bad tree, k or out pointer");
    *placement = k > 16 ? large_k_list_of(t, k) : KDT_LIST_SHARED;
    return KDT_OK;
}

int kdt_tuned_params(const kdt_tree *t, int k, int *stage_levels, int *claim_steps, int *inline_depth,
                     int *light_run)
{
    if (!t || k < 1 || k > 64)
        return set_error(KDT_EINVAL, "bad tree or k");
    if (stage_levels)
        *stage_levels = stage_levels_for(t, k);
    if (claim_steps)
        *claim_steps = claim_steps_for(t, k);
    if (inline_depth)
        *inline_depth = inline_depth_for(t, k);
    if (light_run)
        *light_run = light_run_for(t, k);
    return KDT_OK;
}

// Coordinate search: inline depth, light run, then claim steps, then staging depth, each
// over its candidates with the others at their best so far; every candidate is
// timed over two launches on up to 2^20 of the queries after one warm-up, and
// replaces the best so far only if it is faster by a margin (2 %; 5 % for
// staging, whose cost in occupancy shows more on long runs than on a sample).
// Staging is limited to 8 levels (4 KB), which leaves occupancy unchanged.
int kdt_autotune(kdt_tree *t, const float *d_q, int64_t Q, int k, int flags, int *best_levels, float *best_ms,
                 void *stream)
{
    if (!t || !d_q || Q < 1 || k < 1 || k > 64)
        return set_error(KDT_EINVAL, "bad autotune arguments");
    if (flags & (KDT_LEARNED | KDT_PLAIN_STEP | KDT_CLOSE_FIRST | KDT_STACK))
        return set_error(KDT_EINVAL, "autotune the plain traversal (no KDT_LEARNED, no ablation)");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = Q < ((int64_t)1 << 20) ? Q : ((int64_t)1 << 20);
    int32_t *ids = nullptr;
    float *d2 = nullptr;
    KDT_CUDA(cudaMallocAsync(&ids, (size_t)n * k * 4, s));
    KDT_CUDA(cudaMallocAsync(&d2, (size_t)n * k * 4, s));
    cudaEvent_t e0, e1;
    KDT_CUDA(cudaEventCreate(&e0));
    KDT_CUDA(cudaEventCreate(&e1));
    const int saved_stage = t->stage_levels, saved_claim = t->claim_steps, saved_inline = t->inline_depth;
    const int saved_light = t->light_run, saved_list = t->large_k_list;
    Tuned best{DEFAULT_STAGE_LEVELS, default_claim_steps(k), DEFAULT_INLINE_DEPTH, DEFAULT_LIGHT_RUN,
               DEFAULT_LARGE_K_LIST};
    float best_t = 3.4e38f;
    int rc = KDT_OK;
    auto measure = [&](const Tuned &c, float *out) {
        t->stage_levels = c.stage_levels;
        t->claim_steps = c.claim_steps;
        t->inline_depth = c.inline_depth;
        t->light_run = c.light_run;
        t->large_k_list = c.large_k_list;
        for (int rep = 0; rep < 3 && rc == KDT_OK; ++rep) {
            rc = run_query(t, d_q, n, k, INFINITY, flags & ~KDT_NO_STAGE, MODE_RESULTS, ids, d2, nullptr, s);
            if (rc == KDT_OK && rep == 0)
                rc = cudaEventRecord(e0, s) == cudaSuccess ? KDT_OK : set_error(KDT_ECUDA, "event record");
        }
        float ms = 0.f;
        if (rc == KDT_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = set_error(KDT_ECUDA, "event timing failed");
        *out = ms * 0.5f;  // two timed launches
        return rc == KDT_OK;
    };
    auto consider = [&](Tuned c, float margin) {
        float ms;
        if (measure(c, &ms) && ms < best_t * (1.f - margin)) {
            best_t = ms;
            best = c;
        }
    };
    const bool simple_ok = !(flags & KDT_UNORDERED) && k <= 16 && t->layout != 2;
    consider(best, 0.f);
    if (k > 16 && rc == KDT_OK) {
        // the heap placement follows the queries' length, not a timing: on a
        // sample this size the launch's tail of a few long queries decides,
        // where fewer, less contended warps win, while at full size the
        // global heap's residency does (clustered 2^24, k = 32 / 64: 1.6x).
        // Long queries amortise the heap's trips to memory, short ones do not
        // (surface k = 32, ~190 nodes per query: the shared heap is 1.6x
        // faster).  Threshold: 1024 processed nodes per query.
        rc = run_query(t, d_q, n, k, INFINITY, flags & ~KDT_NO_STAGE, MODE_VISITS, nullptr, nullptr, ids, s);
        std::vector<int32_t> hv(n);
        if (rc == KDT_OK && (cudaMemcpyAsync(hv.data(), ids, (size_t)n * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                             cudaStreamSynchronize(s) != cudaSuccess))
            rc = set_error(KDT_ECUDA, "visit count copy failed");
        double sum = 0.0;
        for (int32_t v : hv)
            sum += v;
        if (rc == KDT_OK && sum >= 1024.0 * (double)n) {
            best.large_k_list = KDT_LIST_GLOBAL;
            float ms;
            if (measure(best, &ms))  // the reference time of the later candidates
                best_t = ms;
        }
    }
    for (int d : {3, 4, 1, 0}) {
        Tuned c = best;
        c.inline_depth = d;
        if (rc == KDT_OK && (d > 0 || simple_ok))
            consider(c, 0.02f);
    }
    for (int lr : {4, 8}) {
        Tuned c = best;
        c.light_run = lr;
        if (rc == KDT_OK && best.inline_depth > 0)
            consider(c, 0.02f);
    }
    for (int cs : {16, 32, 64, 128}) {
        Tuned c = best;
        c.claim_steps = cs;
        if (rc == KDT_OK && cs != best.claim_steps)
            consider(c, 0.02f);
    }
    if (best.inline_depth > 0) {
        for (int lv : {4, 6, 8}) {
            Tuned c = best;
            c.stage_levels = lv;
            if (rc == KDT_OK && stage_fits(t, lv, 64 * 1024))
                consider(c, 0.05f);
        }
    }
    t->stage_levels = saved_stage;
    t->claim_steps = saved_claim;
    t->inline_depth = saved_inline;
    t->light_run = saved_light;
    t->large_k_list = saved_list;
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
        *best_levels = best.stage_levels;
    if (best_ms)
        *best_ms = best_t;
    return KDT_OK;
}

int kdt_tuning_save(const char *path)
{
    if (!path)
        return set_error(KDT_EINVAL, "path is NULL");
    std::vector<std::pair<ShapeKey, Tuned>> rows;
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
        const Tuned &v = rows[i].second;
        ok = fprintf(f,
                     "  {\"gpu\": \"%s\", \"D\": %d, \"k_bucket\": %d, \"log2n\": %d, \"stage_levels\": %d, "
                     "\"claim_steps\": %d, \"inline_depth\": %d, \"light_run\": %d, \"large_k_list\": %d}%s\n",
                     std::get<0>(key).c_str(), std::get<1>(key), std::get<2>(key), std::get<3>(key), v.stage_levels,
                     v.claim_steps, v.inline_depth, v.light_run, v.large_k_list, i + 1 < rows.size() ? "," : "") > 0;
    }
    ok = ok && fprintf(f, "]\n") > 0;
    ok = (fclose(f) == 0) && ok;
    return ok ? KDT_OK : set_error(KDT_EIO, "write to %s failed", path);
}

// reads the format kdt_tuning_save writes (one object per line); rows without
// claim_steps / inline_depth / light_run take the defaults
int kdt_tuning_load(const char *path)
{
    if (!path)
        return set_error(KDT_EINVAL, "path is NULL");
    FILE *f = fopen(path, "r");
    if (!f)
        return set_error(KDT_EIO, "cannot open %s", path);
    char line[512];
    std::vector<std::pair<ShapeKey, Tuned>> rows;
    bool bad = false;
    while (fgets(line, sizeof line, f)) {
        const char *g = strstr(line, "\"gpu\": \"");
        if (!g)
            continue;
        g += 8;
        const char *ge = strchr(g, '"');
        int D, kb, l2, lv, cs = -1, inl = -1, lr = -1, kl = -1;
        if (!ge || sscanf(ge, "\", \"D\": %d, \"k_bucket\": %d, \"log2n\": %d, \"stage_levels\": %d", &D, &kb, &l2,
                          &lv) != 4 || lv < 0 || lv > 16 || kb < 0 || kb > 5) {
            bad = true;
            break;
        }
        const char *c = strstr(ge, "\"claim_steps\": ");
        const char *d = strstr(ge, "\"inline_depth\": ");
        const char *r = strstr(ge, "\"light_run\": ");
        const char *l = strstr(ge, "\"large_k_list\": ");
        if ((c && (sscanf(c + 15, "%d", &cs) != 1 || cs < 1 || cs > 256)) ||
            (d && (sscanf(d + 16, "%d", &inl) != 1 || inl < 0 || inl > 4)) ||
            (r && (sscanf(r + 13, "%d", &lr) != 1 || lr < 1 || lr > 64)) ||
            (l && (sscanf(l + 16, "%d", &kl) != 1 || kl < 0 || kl > KDT_LIST_GROUP8))) {
            bad = true;
            break;
        }
        const int k_rep = kb == 0 ? 1 : (1 << kb);
        rows.emplace_back(ShapeKey(std::string(g, ge - g), D, kb, l2),
                          Tuned{lv, c ? cs : default_claim_steps(k_rep), d ? inl : DEFAULT_INLINE_DEPTH,
                                r ? lr : DEFAULT_LIGHT_RUN, l ? kl : DEFAULT_LARGE_K_LIST});
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
