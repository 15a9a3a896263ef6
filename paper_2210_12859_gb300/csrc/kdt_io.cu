// Tree files: a built tree saved as its level-order arrays, so that a large
// tree is built once and reloaded without rebuilding.
//
// Layout (little-endian): magic "KDTTREE1", int32 version (2), int32 D,
// int64 N, int32 split mode (0: level mod D, 1: stored per node; absent in
// version 1), float32 coords[N][D] (point at each level-order node), int32
// ids[N] (its input index), uint8 dims[N] (split mode 1 only), float32
// bbox[6], uint64 FNV-1a hash of everything after the magic and before the
// hash.
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

__global__ void import_kernel(const float *__restrict__ coords, const int32_t *__restrict__ ids,
                              const uint8_t *__restrict__ dims, int64_t n, int D, float4 *__restrict__ nodes,
                              int32_t *__restrict__ out_ids)
{
    const int NF = D <= 4 ? 1 : 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        float v[8];
        for (int j = 0; j < 8; ++j)
            v[j] = j < D ? coords[t * D + j] : 0.f;
        if (D <= 3) {
            const uint32_t word = (uint32_t)ids[t] | (dims ? (uint32_t)dims[t] << NODE_DIM_SHIFT : 0u);
            nodes[t] = make_float4(v[0], v[1], v[2], __uint_as_float(word));
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
    const int32_t mode = t->layout == 3 ? 1 : 0;
    std::vector<uint8_t> dims(mode ? N : 0);
    int rc = kdt_tree_export(t, d_coords, d_ids, nullptr);
    if (rc == KDT_OK && mode)
        rc = kdt_tree_split_dims(t, (uint8_t *)d_coords, nullptr) == KDT_OK ? KDT_OK : KDT_ECUDA;
    if (rc == KDT_OK) {
        if (mode) {
            e = cudaMemcpy(dims.data(), d_coords, dims.size(), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && kdt_tree_export(t, d_coords, nullptr, nullptr) != KDT_OK)
                e = cudaErrorUnknown;
        }
        if (e == cudaSuccess)
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
    const int32_t ver = 2, d32 = D;
    Fnv h;
    h.add(&ver, 4);
    h.add(&d32, 4);
    h.add(&N, 8);
    h.add(&mode, 4);
    h.add(coords.data(), coords.size() * 4);
    h.add(ids.data(), ids.size() * 4);
    h.add(dims.data(), dims.size());
    h.add(bbox.data(), 24);
    bool ok = fwrite(TREE_MAGIC, 1, 8, f) == 8 && fwrite(&ver, 4, 1, f) == 1 && fwrite(&d32, 4, 1, f) == 1 &&
              fwrite(&N, 8, 1, f) == 1 && fwrite(&mode, 4, 1, f) == 1 &&
              fwrite(coords.data(), 4, coords.size(), f) == coords.size() &&
              fwrite(ids.data(), 4, ids.size(), f) == ids.size() &&
              fwrite(dims.data(), 1, dims.size(), f) == dims.size() && fwrite(bbox.data(), 4, 6, f) == 6 &&
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
    int32_t ver = 0, D = 0, mode = 0;
    int64_t N = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, TREE_MAGIC, 8) == 0 && fread(&ver, 4, 1, f) == 1 &&
              (ver == 1 || ver == 2) && fread(&D, 4, 1, f) == 1 && fread(&N, 8, 1, f) == 1 && D >= 1 && D <= 8 &&
              N >= 1 && N < ((int64_t)1 << 30);
    if (ok && ver == 2)
        ok = fread(&mode, 4, 1, f) == 1 && (mode == 0 || (mode == 1 && D <= 3));
    std::vector<float> coords, bbox(6);
    std::vector<int32_t> ids;
    std::vector<uint8_t> dims;
    uint64_t stored = 0;
    if (ok) {
        coords.resize((size_t)N * D);
        ids.resize((size_t)N);
        dims.resize(mode ? (size_t)N : 0);
        ok = fread(coords.data(), 4, coords.size(), f) == coords.size() &&
             fread(ids.data(), 4, ids.size(), f) == ids.size() && fread(dims.data(), 1, dims.size(), f) == dims.size() &&
             fread(bbox.data(), 4, 6, f) == 6 && fread(&stored, 8, 1, f) == 1;
    }
    fclose(f);
    if (ok) {
        Fnv h;
        h.add(&ver, 4);
        h.add(&D, 4);
        h.add(&N, 8);
        if (ver == 2)
            h.add(&mode, 4);
        h.add(coords.data(), coords.size() * 4);
        h.add(ids.data(), ids.size() * 4);
        h.add(dims.data(), dims.size());
        h.add(bbox.data(), 24);
        ok = h.h == stored;
    }
    if (ok)
        for (int64_t i = 0; i < N && ok; ++i)
            ok = ids[i] >= 0 && ids[i] < N && (dims.empty() || dims[i] < D);
    if (!ok)
        return set_error(KDT_EIO, "%s is not a tree file of this version (or is damaged)", path);
    kdt_tree *t = nullptr;
    KDT_TRY(kdt_tree_alloc_internal(N, D, &t));
    if (mode)
        t->layout = 3;
    cudaStream_t s = (cudaStream_t)stream;
    float *d_coords = nullptr;
    int32_t *d_ids = nullptr;
    uint8_t *d_dims = nullptr;
    cudaError_t e = cudaMalloc(&d_coords, coords.size() * 4);
    if (e == cudaSuccess)
        e = cudaMalloc(&d_ids, ids.size() * 4);
    if (e == cudaSuccess && mode)
        e = cudaMalloc(&d_dims, dims.size());
    if (e == cudaSuccess && mode)
        e = cudaMemcpy(d_dims, dims.data(), dims.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_coords, coords.data(), coords.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_ids, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->bbox, bbox.data(), 24, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        unsigned g = (unsigned)std::min<int64_t>((N + 255) / 256, (int64_t)num_sms() * 16);
        KDT_LAUNCH import_kernel<<<g, 256, 0, s>>>(d_coords, d_ids, d_dims, N, D, t->nodes, t->ids);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
    }
    cudaFree(d_coords);
    cudaFree(d_ids);
    cudaFree(d_dims);
    if (e != cudaSuccess) {
        kdt_free(t);
        return cuda_error(e, "tree upload", __FILE__, __LINE__);
    }
    *out = t;
    return KDT_OK;
}

}  // extern "C"
