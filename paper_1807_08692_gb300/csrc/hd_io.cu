// Checkpoints of the offline artefacts: the normalised graph W (Sec. 3) and
// the eigenpairs (Sec. 4.1), which the paper stores once and reuses for every
// query.  Flat little-endian files: a 32-byte header, then the device arrays
// as they are stored.
//
//   graph: "HDGRAPH1" | n (i64) | nnz (i64) | reserved (i64)
//          row_ptr i32[n+1] | col i32[nnz] | val f32[nnz] | dinv f32[n]
//   eig:   "HDEIG001" | n (i64) | r (i32) | storage (i32) | ldu (i32) | pad (i32)
//          lambda f64[r] | U (n x ldu elements of the storage type) | scale f32[n] (fp8 only)
#include <cstdio>
#include <cstring>
#include <vector>

#include "hd_internal.cuh"

namespace {

struct File {
    FILE* f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

int write_all(hd_ctx* ctx, FILE* f, const void* p, size_t bytes) {
    if (bytes && fwrite(p, 1, bytes, f) != bytes) return hd_fail(ctx, HD_ERR_INVALID_ARG, "write failed");
    return HD_OK;
}

int read_all(hd_ctx* ctx, FILE* f, void* p, size_t bytes) {
    if (bytes && fread(p, 1, bytes, f) != bytes) return hd_fail(ctx, HD_ERR_INVALID_ARG, "file too short");
    return HD_OK;
}

// device -> file through a host staging buffer
int dev_to_file(hd_ctx* ctx, FILE* f, const void* d, size_t bytes) {
    std::vector<char> h(bytes);
    if (bytes) {
        HD_CUDA(ctx, cudaMemcpyAsync(h.data(), d, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return write_all(ctx, f, h.data(), bytes);
}

int file_to_dev(hd_ctx* ctx, FILE* f, void* d, size_t bytes) {
    std::vector<char> h(bytes);
    int rc = read_all(ctx, f, h.data(), bytes);
    if (rc) return rc;
    if (bytes) {
        HD_CUDA(ctx, cudaMemcpyAsync(d, h.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
        HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return HD_OK;
}

size_t elem_bytes(int storage) { return storage == HD_F32 ? 4 : storage == HD_BF16 ? 2 : 1; }

}  // namespace

extern "C" {

int hd_graph_save(hd_ctx* ctx, const hd_graph* g, const char* path) {
    if (!ctx || !g || !path) return HD_ERR_INVALID_ARG;
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    File F;
    F.f = fopen(path, "wb");
    if (!F.f) return hd_fail(ctx, HD_ERR_INVALID_ARG, "cannot open %s for writing", path);
    const int64_t hdr[3] = {g->n, g->nnz, 0};
    int rc = write_all(ctx, F.f, "HDGRAPH1", 8);
    if (!rc) rc = write_all(ctx, F.f, hdr, sizeof hdr);
    if (!rc) rc = dev_to_file(ctx, F.f, g->row_ptr, (size_t)(g->n + 1) * 4);
    if (!rc) rc = dev_to_file(ctx, F.f, g->col, (size_t)g->nnz * 4);
    if (!rc) rc = dev_to_file(ctx, F.f, g->val, (size_t)g->nnz * 4);
    if (!rc) rc = dev_to_file(ctx, F.f, g->dinv, (size_t)g->n * 4);
    return rc;
}

int hd_graph_load(hd_ctx* ctx, const char* path, hd_graph** out) {
    if (!ctx || !path || !out) return HD_ERR_INVALID_ARG;
    *out = nullptr;
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    File F;
    F.f = fopen(path, "rb");
    if (!F.f) return hd_fail(ctx, HD_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8];
    int64_t hdr[3];
    int rc = read_all(ctx, F.f, magic, 8);
    if (!rc) rc = read_all(ctx, F.f, hdr, sizeof hdr);
    if (rc) return rc;
    if (memcmp(magic, "HDGRAPH1", 8) || hdr[0] <= 0 || hdr[1] < 0 || hdr[1] >= ((int64_t)1 << 31))
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "%s is not a graph checkpoint", path);
    hd_graph* g = nullptr;
    rc = hd_graph_alloc_internal(ctx, hdr[0], hdr[1], &g);
    if (rc) return rc;
    rc = file_to_dev(ctx, F.f, g->row_ptr, (size_t)(g->n + 1) * 4);
    if (!rc) rc = file_to_dev(ctx, F.f, g->col, (size_t)g->nnz * 4);
    if (!rc) rc = file_to_dev(ctx, F.f, g->val, (size_t)g->nnz * 4);
    if (!rc) rc = file_to_dev(ctx, F.f, g->dinv, (size_t)g->n * 4);
    if (!rc) rc = hd_graph_check(ctx, g);
    if (rc) {
        hd_graph_destroy(g);
        return rc;
    }
    *out = g;
    return HD_OK;
}

int hd_eig_save(hd_ctx* ctx, const hd_eig* e, const char* path) {
    if (!ctx || !e || !path) return HD_ERR_INVALID_ARG;
    if (e->sparse) return hd_fail(ctx, HD_ERR_INVALID_ARG, "sparsified eigenpairs are not saved (sparsify on load)");
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    File F;
    F.f = fopen(path, "wb");
    if (!F.f) return hd_fail(ctx, HD_ERR_INVALID_ARG, "cannot open %s for writing", path);
    const int64_t n = e->n;
    const int32_t meta[4] = {e->r, e->storage, e->ldu, 0};
    int rc = write_all(ctx, F.f, "HDEIG001", 8);
    if (!rc) rc = write_all(ctx, F.f, &n, 8);
    if (!rc) rc = write_all(ctx, F.f, meta, sizeof meta);
    if (!rc) rc = write_all(ctx, F.f, e->lambda_h.data(), (size_t)e->r * 8);
    if (!rc) rc = dev_to_file(ctx, F.f, e->U, (size_t)n * e->ldu * elem_bytes(e->storage));
    if (!rc && e->storage == HD_FP8) rc = dev_to_file(ctx, F.f, e->scale, (size_t)n * 4);
    return rc;
}

int hd_eig_load(hd_ctx* ctx, const char* path, hd_eig** out) {
    if (!ctx || !path || !out) return HD_ERR_INVALID_ARG;
    *out = nullptr;
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    File F;
    F.f = fopen(path, "rb");
    if (!F.f) return hd_fail(ctx, HD_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8];
    int64_t n = 0;
    int32_t meta[4];
    int rc = read_all(ctx, F.f, magic, 8);
    if (!rc) rc = read_all(ctx, F.f, &n, 8);
    if (!rc) rc = read_all(ctx, F.f, meta, sizeof meta);
    if (rc) return rc;
    const int32_t r = meta[0], storage = meta[1], ldu = meta[2];
    const int32_t want_ldu = r > 0 ? (r + 15) / 16 * 16 : 16;
    if (memcmp(magic, "HDEIG001", 8) || n <= 0 || r < 0 || r > 1024 ||
        (storage != HD_F32 && storage != HD_BF16 && storage != HD_FP8) || ldu != want_ldu)
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "%s is not an eigenpair checkpoint", path);
    hd_eig* e = nullptr;
    rc = hd_eig_alloc(ctx, n, r, storage, &e);
    if (rc) return rc;
    e->lambda_h.resize(r);
    rc = read_all(ctx, F.f, e->lambda_h.data(), (size_t)r * 8);
    if (!rc && r > 0) {
        rc = hd_check_cuda(ctx, cudaMemcpyAsync(e->lambda_d, e->lambda_h.data(), (size_t)r * 8,
                                                cudaMemcpyHostToDevice, ctx->stream), "lambda", __FILE__, __LINE__);
    }
    if (!rc) rc = file_to_dev(ctx, F.f, e->U, (size_t)n * ldu * elem_bytes(storage));
    if (!rc && storage == HD_FP8) rc = file_to_dev(ctx, F.f, e->scale, (size_t)n * 4);
    // the bf16 [hi | lo] copy of fp32 storage is derived, not stored
    if (!rc && storage == HD_F32 && r > 0) rc = hd_eig_store_from_device_f32(ctx, e, (const float*)e->U, ldu);
    if (!rc) rc = hd_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "eig load", __FILE__, __LINE__);
    if (rc) {
        hd_eig_destroy(e);
        return rc;
    }
    *out = e;
    return HD_OK;
}

}  // extern "C"
