// Tree files: a built tree saved as its level-order arrays, so that a large
// tree is built once and reloaded without rebuilding.
//
// Layout (little-endian): magic "KDTTREE1", int32 version 1, int32 D,
// int64 N, float32 coords[N][D] (point at each level-order node), int32
// ids[N] (its input index), float32 bbox[6], uint64 FNV-1a hash of everything
// after the magic and before the hash.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "kdt_query.cuh"

namespace kdt {
namespace {

const char TREE_MAGIC[8] = {'K', 'D', 'T', 'T', 'R', 'E', 'E', '1'};

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n)
    {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
};

__global__ void import_kernel(const float *__restrict__ coords, const int32_t *__restrict__ ids, int64_t n, int D,
                              float4 *__restrict__ nodes, int32_t *__restrict__ out_ids)
{
    const int NF = D <= 4 ? 1 : 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        float v[8];
        for (int j = 0; j < 8; ++j)
            v[j] = j < D ? coords[t * D + j] : 0.f;
        if (D <= 3) {
            nodes[t] = make_float4(v[0], v[1], v[2], __int_as_float(ids[t]));
        } else {
            nodes[t * NF] = make_float4(v[0], v[1], v[2], v[3]);
            if (NF == 2)
                nodes[t * NF + 1] = make_float4(v[4], v[5], v[6], v[7]);
            out_ids[t] = ids[t];
        }
    }
}

}  // namespace
}  // namespace kdt

using namespace kdt;

extern "C" {

int kdt_tree_save(const kdt_tree *t, const char *path)
{
    if (!t || !path)
        return set_error(KDT_EINVAL, "NULL tree or path");
    const int64_t N = t->N;
    const int D = t->D;
    float *d_coords = nullptr;
    int32_t *d_ids = nullptr;
    KDT_CUDA(cudaMalloc(&d_coords, (size_t)N * D * 4));
    cudaError_t e = cudaMalloc(&d_ids, (size_t)N * 4);
    if (e != cudaSuccess) {
        cudaFree(d_coords);
        return cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
    }
    std::vector<float> coords((size_t)N * D), bbox(6);
    std::vector<int32_t> ids(N);
    int rc = kdt_tree_export(t, d_coords, d_ids, nullptr);
    if (rc == KDT_OK) {
        e = cudaMemcpy(coords.data(), d_coords, coords.size() * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(ids.data(), d_ids, ids.size() * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(bbox.data(), t->bbox, 24, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            rc = cuda_error(e, "tree download", __FILE__, __LINE__);
    }
    cudaFree(d_coords);
    cudaFree(d_ids);
    if (rc != KDT_OK)
        return rc;
    FILE *f = fopen(path, "wb");
    if (!f)
        return set_error(KDT_EIO, "cannot open %s for writing", path);
    const int32_t ver = 1, d32 = D;
    Fnv h;
    h.add(&ver, 4);
    h.add(&d32, 4);
    h.add(&N, 8);
    h.add(coords.data(), coords.size() * 4);
    h.add(ids.data(), ids.size() * 4);
    h.add(bbox.data(), 24);
    bool ok = fwrite(TREE_MAGIC, 1, 8, f) == 8 && fwrite(&ver, 4, 1, f) == 1 && fwrite(&d32, 4, 1, f) == 1 &&
              fwrite(&N, 8, 1, f) == 1 && fwrite(coords.data(), 4, coords.size(), f) == coords.size() &&
              fwrite(ids.data(), 4, ids.size(), f) == ids.size() && fwrite(bbox.data(), 4, 6, f) == 6 &&
              fwrite(&h.h, 8, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    return ok ? KDT_OK : set_error(KDT_EIO, "write to %s failed", path);
}

int kdt_tree_load(const char *path, void *stream, kdt_tree **out)
{
    if (!path || !out)
        return set_error(KDT_EINVAL, "NULL path or out");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f)
        return set_error(KDT_EIO, "cannot open %s", path);
    char magic[8];
    int32_t ver = 0, D = 0;
    int64_t N = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, TREE_MAGIC, 8) == 0 && fread(&ver, 4, 1, f) == 1 &&
              ver == 1 && fread(&D, 4, 1, f) == 1 && fread(&N, 8, 1, f) == 1 && D >= 1 && D <= 8 && N >= 1 &&
              N < ((int64_t)1 << 30);
    std::vector<float> coords, bbox(6);
    std::vector<int32_t> ids;
    uint64_t stored = 0;
    if (ok) {
        coords.resize((size_t)N * D);
        ids.resize((size_t)N);
        ok = fread(coords.data(), 4, coords.size(), f) == coords.size() &&
             fread(ids.data(), 4, ids.size(), f) == ids.size() && fread(bbox.data(), 4, 6, f) == 6 &&
             fread(&stored, 8, 1, f) == 1;
    }
    fclose(f);
    if (ok) {
        Fnv h;
        h.add(&ver, 4);
        h.add(&D, 4);
        h.add(&N, 8);
        h.add(coords.data(), coords.size() * 4);
        h.add(ids.data(), ids.size() * 4);
        h.add(bbox.data(), 24);
        ok = h.h == stored;
    }
    if (ok)
        for (int64_t i = 0; i < N && ok; ++i)
            ok = ids[i] >= 0 && ids[i] < N;
    if (!ok)
        return set_error(KDT_EIO, "%s is not a tree file of this version (or is damaged)", path);
    kdt_tree *t = nullptr;
    KDT_TRY(kdt_tree_alloc_internal(N, D, &t));
    cudaStream_t s = (cudaStream_t)stream;
    float *d_coords = nullptr;
    int32_t *d_ids = nullptr;
    cudaError_t e = cudaMalloc(&d_coords, coords.size() * 4);
    if (e == cudaSuccess)
        e = cudaMalloc(&d_ids, ids.size() * 4);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_coords, coords.data(), coords.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_ids, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->bbox, bbox.data(), 24, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        unsigned g = (unsigned)std::min<int64_t>((N + 255) / 256, (int64_t)num_sms() * 16);
        KDT_LAUNCH import_kernel<<<g, 256, 0, s>>>(d_coords, d_ids, N, D, t->nodes, t->ids);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
    }
    cudaFree(d_coords);
    cudaFree(d_ids);
    if (e != cudaSuccess) {
        kdt_free(t);
        return cuda_error(e, "tree upload", __FILE__, __LINE__);
    }
    *out = t;
    return KDT_OK;
}

}  // extern "C"
