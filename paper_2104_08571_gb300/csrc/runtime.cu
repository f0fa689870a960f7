// C-ABI runtime: contexts, fields, tensor maps, upload/download and the
// Euler step driver.  No kernel arithmetic lives here.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "runtime.h"

namespace ripple {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

ripple_status fail(ripple_status st, const std::string& msg)
{
    set_error(msg);
    return st;
}

ripple_status cuda_fail(cudaError_t e, const char* what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RIPPLE_ERR_OOM : RIPPLE_ERR_CUDA;
}

size_t elem_size(ripple_dtype d) { return d == RIPPLE_F64 ? 8 : 4; }

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool budget_reserve(ripple_ctx ctx, size_t bytes)
{
    size_t cur = ctx->used.load();
    for (;;) {
        if (ctx->budget && cur + bytes > ctx->budget) return false;
        if (ctx->used.compare_exchange_weak(cur, cur + bytes)) return true;
    }
}

FieldGeom make_field_geom(int ndim, const int64_t* dims, int ncomp, ripple_layout layout, int halo,
                          ripple_dtype dtype, size_t* bytes)
{
    const int es = (int)elem_size(dtype);
    const int a = 16 / es;  // 16-byte x alignment in cells
    FieldGeom g{};
    g.ndim = ndim;
    g.ncomp = ncomp;
    g.h = halo;
    g.lead = (a - halo % a) % a;
    for (int d = 0; d < 3; ++d) g.n[d] = d < ndim ? (int)dims[d] : 1;
    g.px = (long long)round_up((size_t)(g.lead + g.n[0] + 2 * halo), (size_t)a);
    g.py = g.n[1] + 2 * halo;
    g.pz = ndim == 3 ? g.n[2] + 2 * halo : 1;
    const long long ncell = g.px * g.py * g.pz;
    if (layout == RIPPLE_SOA) {
        g.cell_stride = 1;
        g.comp_stride = ncell;
    } else {
        g.cell_stride = ncomp;
        g.comp_stride = 1;
    }
    if (bytes) *bytes = round_up((size_t)ncell * ncomp * es, 256);
    return g;
}

bool fault_injected(const char* step)
{
    const char* env = std::getenv("RIPPLE_FAULT");
    if (!env || !*env) return false;
    const size_t n = std::strlen(step);
    for (const char* p = env; *p;) {
        const char* e = std::strchr(p, ',');
        const size_t len = e ? (size_t)(e - p) : std::strlen(p);
        if (len == n && std::strncmp(p, step, n) == 0) return true;
        if (!e) break;
        p = e + 1;
    }
    return false;
}

ripple_status ctx_alloc(ripple_ctx ctx, size_t bytes, void** out)
{
    *out = nullptr;
    if (fault_injected("alloc")) return fail(RIPPLE_ERR_OOM, "device allocation failed (injected: RIPPLE_FAULT=alloc)");
    bytes = round_up(std::max<size_t>(bytes, 256), 256);
    if (!budget_reserve(ctx, bytes))
        return fail(RIPPLE_ERR_BUDGET, "allocation of " + std::to_string(bytes) + " bytes exceeds the memory budget");
    void* p = nullptr;
    if (ctx->alloc_fn) {
        p = ctx->alloc_fn(bytes, ctx->alloc_user);
        if (!p) {
            ctx->used -= bytes;
            return fail(RIPPLE_ERR_OOM, "allocator callback returned NULL");
        }
        if (reinterpret_cast<uintptr_t>(p) % 256) {
            ctx->free_fn(p, ctx->alloc_user);
            ctx->used -= bytes;
            return fail(RIPPLE_ERR_INTERNAL, "allocator callback returned memory not aligned to 256 bytes");
        }
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            ctx->used -= bytes;
            return cuda_fail(e, "cudaMalloc");
        }
    }
    *out = p;
    return RIPPLE_OK;
}

void ctx_free(ripple_ctx ctx, void* p, size_t bytes)
{
    if (!p) return;
    bytes = round_up(std::max<size_t>(bytes, 256), 256);
    if (ctx->alloc_fn) ctx->free_fn(p, ctx->alloc_user);
    else cudaFree(p);
    ctx->used -= bytes;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

ripple_status encode_plane_map(void* buffer, const FieldGeom& g, ripple_layout layout, ripple_dtype dtype, int kind,
                               int r, int tx, int ty, CUtensorMap* out)
{
    auto enc = encode_fn();
    if (!enc) return fail(RIPPLE_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const int es = (int)elem_size(dtype);
    const int nc = g.ncomp;
    const bool soa = layout == RIPPLE_SOA;
    cuuint64_t dims[4], strides[3];
    cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
    cuuint32_t rank;
    char* base = static_cast<char*>(buffer);
    const BoxGeom bg = plane_box(es, nc, !soa, r, tx, ty);
    if (kind == 2) {
        // AoS plane staging of the row kernel: each row viewed as groups of
        // four cells (4 x ncomp elements, a multiple of 16 bytes), so a box
        // as wide as the row tile fits the 256-element box limit per dimension
        if (soa || g.ndim != 3 || g.px % 4 != 0 || bg.bx % 4 != 0)
            return fail(RIPPLE_ERR_INTERNAL, "grouped AoS plane map needs a 3D AoS field");
        rank = 4;
        dims[0] = 4 * nc; dims[1] = g.px / 4; dims[2] = g.py; dims[3] = g.pz;
        strides[0] = 4 * nc * es; strides[1] = g.px * nc * es; strides[2] = g.px * nc * g.py * es;
        box[0] = 4 * nc; box[1] = bg.bx / 4; box[2] = bg.by; box[3] = 1;
    } else if (kind == 0) {
        if (soa) {
            dims[0] = g.px; dims[1] = g.py;
            strides[0] = g.px * es; strides[1] = g.px * g.py * es;
            box[0] = bg.bx; box[1] = bg.by;
            if (g.ndim == 3) {
                rank = 4;
                dims[2] = g.pz; dims[3] = nc;
                strides[2] = g.px * g.py * g.pz * es;
                box[2] = 1; box[3] = nc;
            } else {
                rank = 3;
                dims[2] = nc;
                box[2] = nc;
            }
        } else {
            dims[0] = g.px * nc; dims[1] = g.py;
            strides[0] = g.px * nc * es;
            box[0] = bg.bx * nc; box[1] = bg.by;
            if (g.ndim == 3) {
                rank = 3;
                dims[2] = g.pz;
                strides[1] = g.px * nc * g.py * es;
                box[2] = 1;
            } else {
                rank = 2;
            }
        }
    } else {
        base += geom_elem(g, 0, 0, 0, 0) * es;
        if (soa) {
            dims[0] = g.n[0]; dims[1] = g.n[1];
            strides[0] = g.px * es; strides[1] = g.px * g.py * es;
            box[0] = tx; box[1] = ty;
            if (g.ndim == 3) {
                rank = 4;
                dims[2] = g.n[2]; dims[3] = nc;
                strides[2] = g.px * g.py * g.pz * es;
                box[2] = 1; box[3] = nc;
            } else {
                rank = 3;
                dims[2] = nc;
                box[2] = nc;
            }
        } else {
            dims[0] = (cuuint64_t)g.n[0] * nc; dims[1] = g.n[1];
            strides[0] = g.px * nc * es;
            box[0] = tx * nc; box[1] = ty;
            if (g.ndim == 3) {
                rank = 3;
                dims[2] = g.n[2];
                strides[1] = g.px * nc * g.py * es;
                box[2] = 1;
            } else {
                rank = 2;
            }
        }
    }
    CUresult cr = enc(out, dtype == RIPPLE_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                      rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      // staging loads read NaN beyond the tensor (as the padded cells of an Euler
                      // field); stores are clipped and fill nothing
                      kind != 1 ? CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA : CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS)
        return fail(RIPPLE_ERR_CUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)cr) + ")");
    return RIPPLE_OK;
}

const CUtensorMap* field_map(ripple_field f, int buffer, int kind, int r, int tx, int ty, ripple_status* st)
{
    *st = RIPPLE_OK;
    for (auto& m : f->maps)
        if (m.buffer == buffer && m.kind == kind && m.r == r && m.tx == tx && m.ty == ty) return &m.map;
    MapEntry e{};
    e.buffer = buffer; e.kind = kind; e.r = r; e.tx = tx; e.ty = ty;
    *st = encode_plane_map(f->buf[buffer], f->geom, f->layout, f->dtype, kind, r, tx, ty, &e.map);
    if (*st != RIPPLE_OK) return nullptr;
    f->maps.push_back(e);
    return &f->maps.back().map;
}

ripple_status ensure_second_buffer(ripple_field f)
{
    if (f->buf[1]) return RIPPLE_OK;
    void* p = nullptr;
    ripple_status st = ctx_alloc(f->ctx, f->bytes, &p);
    if (st != RIPPLE_OK) return st;
    RIPPLE_CUDA(cudaMemsetAsync(p, 0, f->bytes, f->ctx->stream));
    f->buf[1] = p;
    f->maps.clear();  // vector may reallocate: entries are re-encoded on demand
    return RIPPLE_OK;
}

static ripple_status map_dev_err(unsigned err, const FieldCtl* host = nullptr)
{
    if (err & DEV_ERR_INTERNAL) return fail(RIPPLE_ERR_INTERNAL, "device-side invariant violated");
    if (err & DEV_ERR_BARRIER) return fail(RIPPLE_ERR_TIMEOUT, "a device-side grid barrier wait ran out");
    if (err & DEV_ERR_TIMEOUT) return fail(RIPPLE_ERR_TIMEOUT, "a device-side bounded wait ran out");
    if (err & DEV_ERR_NUMERIC) {
        std::string msg = "non-positive or NaN density/pressure produced";
        if (host && host->counters[4] > 0) {
            const long long c = host->counters[4];
            const char* what = c == BAD_CELL    ? "updated cell"
                               : c == BAD_INPUT ? "input cell"
                                                : "reconstructed/predicted/face state in the tile starting at cell";
            msg += std::string(" (first at ") + what + " (" + std::to_string(host->counters[5]) + ", " +
                   std::to_string(host->counters[6]) + ", " + std::to_string(host->counters[7]) + "))";
        }
        return fail(RIPPLE_ERR_NUMERIC, msg);
    }
    return RIPPLE_OK;
}

ripple_status take_device_error(ripple_field f)
{
    unsigned err = 0;
    RIPPLE_CUDA(cudaMemcpyAsync(&err, &f->ctl->err, sizeof(unsigned), cudaMemcpyDeviceToHost, f->ctx->stream));
    RIPPLE_CUDA(cudaStreamSynchronize(f->ctx->stream));
    if (err) RIPPLE_CUDA(cudaMemsetAsync(&f->ctl->err, 0, sizeof(unsigned), f->ctx->stream));
    return map_dev_err(err);
}

static int grid_for(ripple_ctx ctx, long long work, int per_block)
{
    long long b = (work + per_block - 1) / per_block;
    long long cap = (long long)ctx->sm_count * 8;
    return (int)std::max<long long>(1, std::min(b, cap));
}

// Euler step dispatch -------------------------------------------------------

cudaError_t sweep_launch(ripple_dtype dt, int dim, int layout, int scheme, int v, const SweepLaunch& L)
{
    if (dt == RIPPLE_F32) return dim == 2 ? sweep_launch_f32_2d(layout, scheme, v, L) : sweep_launch_f32_3d(layout, scheme, v, L);
    return dim == 2 ? sweep_launch_f64_2d(layout, scheme, v, L) : sweep_launch_f64_3d(layout, scheme, v, L);
}
int sweep_smem(ripple_dtype dt, int dim, int layout, int scheme, int v)
{
    if (dt == RIPPLE_F32) return dim == 2 ? sweep_smem_f32_2d(layout, scheme, v) : sweep_smem_f32_3d(layout, scheme, v);
    return dim == 2 ? sweep_smem_f64_2d(layout, scheme, v) : sweep_smem_f64_3d(layout, scheme, v);
}
int sweep_occ(ripple_dtype dt, int dim, int layout, int scheme, int v)
{
    if (dt == RIPPLE_F32) return dim == 2 ? sweep_occ_f32_2d(layout, scheme, v) : sweep_occ_f32_3d(layout, scheme, v);
    return dim == 2 ? sweep_occ_f64_2d(layout, scheme, v) : sweep_occ_f64_3d(layout, scheme, v);
}

}  // namespace ripple

using namespace ripple;

extern "C" {

const char* ripple_last_error(void) { return g_last_error.c_str(); }

const char* ripple_version(void) { return "ripple-gb300 0.1 (sm_103a)"; }

ripple_status ripple_ctx_create(int device, size_t mem_budget_bytes, ripple_ctx* out)
{
    if (!out) return fail(RIPPLE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int n = 0;
    RIPPLE_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(RIPPLE_ERR_INVALID, "no such CUDA device");
    RIPPLE_CUDA(cudaSetDevice(device));
    auto* c = new (std::nothrow) ripple_ctx_s();
    if (!c) return fail(RIPPLE_ERR_OOM, "host allocation failed");
    c->device = device;
    c->budget = mem_budget_bytes;
    cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "ripple_ctx_create");
    }
    c->stream = c->own_stream;
    *out = c;
    return RIPPLE_OK;
}

ripple_status ripple_ctx_destroy(ripple_ctx ctx)
{
    if (!ctx) return RIPPLE_OK;
    if (ctx->nfields.load() != 0) return fail(RIPPLE_ERR_INVALID, "destroy all fields before their context");
    batch_runtime_destroy(ctx);
    cudaStreamSynchronize(ctx->stream);
    ctx_free(ctx, ctx->staging, ctx->staging_bytes);
    ctx_free(ctx, ctx->partials, ctx->partials_bytes);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return RIPPLE_OK;
}

ripple_status ripple_set_stream(ripple_ctx ctx, void* cuda_stream)
{
    if (!ctx) return fail(RIPPLE_ERR_INVALID, "ctx is NULL");
    ctx->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->own_stream;
    return RIPPLE_OK;
}

ripple_status ripple_set_allocator(ripple_ctx ctx, void* (*alloc)(size_t, void*), void (*release)(void*, void*),
                                   void* user)
{
    if (!ctx) return fail(RIPPLE_ERR_INVALID, "ctx is NULL");
    if (ctx->used.load() != 0) return fail(RIPPLE_ERR_INVALID, "set the allocator before allocating");
    if ((alloc == nullptr) != (release == nullptr)) return fail(RIPPLE_ERR_INVALID, "alloc and release go together");
    ctx->alloc_fn = alloc;
    ctx->free_fn = release;
    ctx->alloc_user = user;
    return RIPPLE_OK;
}

ripple_status ripple_ctx_sync(ripple_ctx ctx)
{
    if (!ctx) return fail(RIPPLE_ERR_INVALID, "ctx is NULL");
    RIPPLE_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<ripple_field> fields;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        fields = ctx->fields;
    }
    ripple_status first = RIPPLE_OK;
    for (ripple_field f : fields) {
        ripple_status st = take_device_error(f);
        if (first == RIPPLE_OK) first = st;
    }
    if (layout_bench_take_error(ctx->stream) && first == RIPPLE_OK)
        first = fail(RIPPLE_ERR_TIMEOUT, "a bounded wait of a staged particle update ran out");
    return first;
}

ripple_status ripple_ctx_mem_used(ripple_ctx ctx, size_t* bytes)
{
    if (!ctx || !bytes) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    *bytes = ctx->used.load();
    return RIPPLE_OK;
}

ripple_status ripple_field_create(ripple_ctx ctx, int ndim, const int64_t* dims, int ncomp, ripple_layout layout,
                                  int halo, ripple_dtype dtype, ripple_field* out)
{
    if (!out) return fail(RIPPLE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!ctx || !dims) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    if (ndim < 2 || ndim > 3) return fail(RIPPLE_ERR_INVALID, "ndim must be 2 or 3");
    if (ncomp < 1 || ncomp > 5) return fail(RIPPLE_ERR_INVALID, "ncomp must be 1..5");
    if (halo < 0 || halo > 8) return fail(RIPPLE_ERR_INVALID, "halo must be 0..8");
    if (layout != RIPPLE_AOS && layout != RIPPLE_SOA) return fail(RIPPLE_ERR_INVALID, "bad layout");
    if (dtype != RIPPLE_F32 && dtype != RIPPLE_F64) return fail(RIPPLE_ERR_INVALID, "bad dtype");
    for (int d = 0; d < ndim; ++d)
        if (dims[d] < 1 || dims[d] > (1 << 20)) return fail(RIPPLE_ERR_INVALID, "dims out of range");
    auto* f = new (std::nothrow) ripple_field_s();
    if (!f) return fail(RIPPLE_ERR_OOM, "host allocation failed");
    f->ctx = ctx;
    f->ndim = ndim;
    f->ncomp = ncomp;
    f->halo = halo;
    f->layout = layout;
    f->dtype = dtype;
    f->geom = make_field_geom(ndim, dims, ncomp, layout, halo, dtype, &f->bytes);
    const FieldGeom& g = f->geom;
    // at most 2^32 padded cells per buffer: byte counts stay far from overflow
    // and every tile, item and table count of the kernels fits in 32 bits
    if (g.px * g.py * g.pz > (1LL << 32)) {
        delete f;
        return fail(RIPPLE_ERR_INVALID, "field too large: more than 2^32 padded cells per buffer");
    }
    f->elems = (size_t)(g.px * g.py * g.pz) * ncomp;
    ripple_status st = ctx_alloc(ctx, f->bytes, &f->buf[0]);
    if (st == RIPPLE_OK) st = ctx_alloc(ctx, sizeof(FieldCtl), reinterpret_cast<void**>(&f->ctl));
    if (st != RIPPLE_OK) {
        ctx_free(ctx, f->buf[0], f->bytes);
        delete f;
        return st;
    }
    cudaError_t e = cudaMemsetAsync(f->buf[0], 0, f->bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->ctl, 0, sizeof(FieldCtl), ctx->stream);
    if (e != cudaSuccess) {
        ctx_free(ctx, f->buf[0], f->bytes);
        ctx_free(ctx, f->ctl, sizeof(FieldCtl));
        delete f;
        return cuda_fail(e, "cudaMemsetAsync");
    }
    ctx->nfields++;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->fields.push_back(f);
    }
    *out = f;
    return RIPPLE_OK;
}

ripple_status ripple_field_destroy(ripple_field f)
{
    if (!f) return RIPPLE_OK;
    ripple_ctx ctx = f->ctx;
    cudaStreamSynchronize(ctx->stream);
    eik_scratch_free(f);
    ctx_free(ctx, f->buf[0], f->bytes);
    ctx_free(ctx, f->buf[1], f->bytes);
    ctx_free(ctx, f->ctl, sizeof(FieldCtl));
    ctx->nfields--;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->fields.erase(std::remove(ctx->fields.begin(), ctx->fields.end(), f), ctx->fields.end());
    }
    delete f;
    return RIPPLE_OK;
}

static ripple_status ensure_staging(ripple_ctx ctx, size_t bytes)
{
    if (ctx->staging_bytes >= bytes) return RIPPLE_OK;
    RIPPLE_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx_free(ctx, ctx->staging, ctx->staging_bytes);
    ctx->staging = nullptr;
    ctx->staging_bytes = 0;
    ripple_status st = ctx_alloc(ctx, bytes, &ctx->staging);
    if (st != RIPPLE_OK) return st;
    ctx->staging_bytes = round_up(bytes, 256);
    return RIPPLE_OK;
}

static size_t interior_bytes(ripple_field f)
{
    const FieldGeom& g = f->geom;
    return (size_t)g.n[0] * g.n[1] * g.n[2] * f->ncomp * elem_size(f->dtype);
}

ripple_status ripple_field_upload_device(ripple_field f, const void* src, ripple_layout src_layout)
{
    if (!f || !src) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    if (src_layout != RIPPLE_AOS && src_layout != RIPPLE_SOA) return fail(RIPPLE_ERR_INVALID, "bad layout");
    const FieldGeom& g = f->geom;
    const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
    RIPPLE_CUDA(launch_interior_copy(f->dtype, f->buf[f->cur], g, const_cast<void*>(src), src_layout, 0,
                                     grid_for(f->ctx, total, 256), f->ctx->stream));
    f->prepared = false;
    return RIPPLE_OK;
}

ripple_status ripple_field_download_device(ripple_field f, void* dst, ripple_layout dst_layout)
{
    if (!f || !dst) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    if (dst_layout != RIPPLE_AOS && dst_layout != RIPPLE_SOA) return fail(RIPPLE_ERR_INVALID, "bad layout");
    const FieldGeom& g = f->geom;
    const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
    RIPPLE_CUDA(launch_interior_copy(f->dtype, f->buf[f->cur], g, dst, dst_layout, 1, grid_for(f->ctx, total, 256),
                                     f->ctx->stream));
    return RIPPLE_OK;
}

ripple_status ripple_field_upload(ripple_field f, const void* src, ripple_layout src_layout)
{
    if (!f || !src) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    const size_t bytes = interior_bytes(f);
    ripple_status st = ensure_staging(f->ctx, bytes);
    if (st != RIPPLE_OK) return st;
    RIPPLE_CUDA(cudaMemcpyAsync(f->ctx->staging, src, bytes, cudaMemcpyHostToDevice, f->ctx->stream));
    st = ripple_field_upload_device(f, f->ctx->staging, src_layout);
    if (st != RIPPLE_OK) return st;
    RIPPLE_CUDA(cudaStreamSynchronize(f->ctx->stream));
    return RIPPLE_OK;
}

ripple_status ripple_field_download(ripple_field f, void* dst, ripple_layout dst_layout)
{
    if (!f || !dst) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    const size_t bytes = interior_bytes(f);
    ripple_status st = ensure_staging(f->ctx, bytes);
    if (st != RIPPLE_OK) return st;
    st = ripple_field_download_device(f, f->ctx->staging, dst_layout);
    if (st != RIPPLE_OK) return st;
    RIPPLE_CUDA(cudaMemcpyAsync(dst, f->ctx->staging, bytes, cudaMemcpyDeviceToHost, f->ctx->stream));
    return take_device_error(f);
}

ripple_status ripple_field_describe(ripple_field f, ripple_field_desc* out)
{
    if (!f || !out) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    const FieldGeom& g = f->geom;
    out->ndim = f->ndim;
    out->ncomp = f->ncomp;
    out->halo = f->halo;
    out->layout = f->layout;
    out->dtype = f->dtype;
    for (int d = 0; d < 3; ++d) out->dims[d] = g.n[d];
    out->padded[0] = g.px;
    out->padded[1] = g.py;
    out->padded[2] = g.pz;
    out->x_lead = g.lead;
    out->buffer_bytes = f->bytes;
    out->current = f->buf[f->cur];
    return RIPPLE_OK;
}

ripple_status ripple_field_set_sweep(ripple_field f, int variant, int zchunk)
{
    if (!f) return fail(RIPPLE_ERR_INVALID, "NULL field");
    if (variant < -1 || variant >= kNumSweepVariants) return fail(RIPPLE_ERR_INVALID, "unknown sweep variant");
    if (zchunk < 0) return fail(RIPPLE_ERR_INVALID, "zchunk must be >= 0");
    f->variant = variant;
    f->zchunk = zchunk;
    return RIPPLE_OK;
}

// Walks of a one-axis sweep (euler_force_walk.cuh): about 16 per resident
// warp, so that the grid-stride walks spread evenly over the SMs, and at least
// 4 chunks (x) or 16 rows (y, z) long, so that the face a walk shares with the
// walk before it (evaluated by both) stays a small part of the arithmetic.
static WalkGeom walk_geom(const FieldGeom& g, int axis, long long resident_warps)
{
    WalkGeom w{};
    w.f = g;
    const long long target = std::max(1LL, 16 * resident_warps);
    const long long nch = (g.n[0] + 63) / 64;
    const long long nyz = (long long)g.n[1] * (g.ndim == 3 ? g.n[2] : 1);  // rows of the x sweep
    if (axis == 0) {
        long long cpw = nch * nyz / target;
        cpw = std::max(std::min(cpw, nch), std::min(4LL, nch));
        w.seg = (int)(64 * cpw);
        w.nseg = (int)((nch + cpw - 1) / cpw);
        w.nstrips = 0;
        w.nlines = 1;
        w.walks = (int)(w.nseg * nyz);
    } else {
        const long long na = g.n[axis];
        const long long lines = g.ndim == 3 ? g.n[axis == 1 ? 2 : 1] : 1;
        long long rows = nch * lines * na / target;
        rows = std::max(std::min(rows, na), std::min(16LL, na));
        w.seg = (int)rows;
        w.nseg = (int)((na + rows - 1) / rows);
        w.nstrips = (int)nch;
        w.nlines = (int)lines;
        w.walks = (int)(w.nseg * nch * lines);
    }
    return w;
}

ripple_status ripple_fv_step(ripple_field U, const ripple_fv_params* p, int64_t nsteps, ripple_fv_stats* stats)
{
    if (!U || !p) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    if (nsteps < 0) return fail(RIPPLE_ERR_INVALID, "nsteps < 0");
    if (U->ncomp != U->ndim + 2) return fail(RIPPLE_ERR_INVALID, "Euler fields need ncomp = ndim + 2");
    if (p->scheme != RIPPLE_RUSANOV1 && p->scheme != RIPPLE_MUSCL_HANCOCK_MINMOD && p->scheme != RIPPLE_FORCE_SPLIT)
        return fail(RIPPLE_ERR_INVALID, "bad scheme");
    if (p->bc != RIPPLE_BC_PERIODIC && p->bc != RIPPLE_BC_TRANSMISSIVE) return fail(RIPPLE_ERR_INVALID, "bad bc");
    const int R = p->scheme == RIPPLE_MUSCL_HANCOCK_MINMOD ? 2 : 1;
    if (U->halo < R) return fail(RIPPLE_ERR_INVALID, "halo smaller than the stencil radius");
    if (!(p->gamma > 1.0) || !(p->cfl > 0.0)) return fail(RIPPLE_ERR_INVALID, "need gamma > 1 and cfl > 0");
    const FieldGeom& g = U->geom;
    for (int d = 0; d < U->ndim; ++d) {
        if (!(p->dx[d] > 0.0)) return fail(RIPPLE_ERR_INVALID, "dx must be > 0");
        if (p->bc == RIPPLE_BC_PERIODIC && g.n[d] < U->halo)
            return fail(RIPPLE_ERR_INVALID, "periodic axes need at least halo cells");
    }
    ripple_ctx ctx = U->ctx;
    ripple_status st = ensure_second_buffer(U);
    if (st != RIPPLE_OK) return st;
    if (!U->pad_nan) {
        // stencil items beyond the ghost layers then read NaN (ignored by the
        // admissibility minimum); prep below refills the current face ghosts
        const long long cells = g.px * g.py * g.pz;
        for (int b = 0; b < 2; ++b)
            RIPPLE_CUDA(launch_pad_nan(U->dtype, U->buf[b], g, grid_for(ctx, cells, 256), ctx->stream));
        U->pad_nan = true;
        U->prepared = false;
    }

    const int layout = U->layout == RIPPLE_SOA ? LAYOUT_SOA : LAYOUT_AOS;
    const int scheme = p->scheme == RIPPLE_MUSCL_HANCOCK_MINMOD ? SCHEME_MUSCL
                       : p->scheme == RIPPLE_FORCE_SPLIT    ? SCHEME_FORCE
                                                            : SCHEME_RUSANOV1;
    const bool split = scheme == SCHEME_FORCE;
    int v = U->variant;
    if (v < 0 || sweep_smem(U->dtype, U->ndim, layout, scheme, v) == 0) {
        // default: the row kernel where it exists (FP32 3D MUSCL-Hancock) for SoA
        // fields, else the packed pair kernel (FP32), else the first that fits.
        // (AoS planes staged in shared memory put a row's cells 20 bytes apart,
        // so the row kernel's per-lane loads of an AoS plane conflict in the
        // shared-memory banks: measured 0.71 against 0.60 ms per 256^3 step for
        // the pair kernel, whose items read AoS planes in a friendlier order.)
        const bool row_ok = layout == LAYOUT_SOA && sweep_smem(U->dtype, U->ndim, layout, scheme, kRowVariant) > 0;
        v = row_ok ? kRowVariant : sweep_smem(U->dtype, U->ndim, layout, scheme, kPairVariant) > 0 ? kPairVariant : -1;
        for (int c = 0; c < kNumSweepVariants && v < 0; ++c)
            if (sweep_smem(U->dtype, U->ndim, layout, scheme, c) > 0) v = c;
        if (v < 0) return fail(RIPPLE_ERR_INTERNAL, "no sweep kernel fits this configuration");
        // a 2D grid with fewer tiles than SMs: the shorter tile spreads it over more SMs
        // (the one-cell-per-item 32x4 variant; FP64 arithmetic is the bound there)
        auto tiles = [&](int c) {
            return ((g.n[0] + kSweepVariants[c].tx - 1) / kSweepVariants[c].tx) *
                   ((g.n[1] + kSweepVariants[c].ty - 1) / kSweepVariants[c].ty);
        };
        if (U->ndim == 2 && U->dtype == RIPPLE_F64 && tiles(v) < ctx->sm_count &&
            sweep_smem(U->dtype, U->ndim, layout, scheme, 1) > 0 && tiles(1) > tiles(v))
            v = 1;
    }
    const int tx = kSweepVariants[v].tx, ty = kSweepVariants[v].ty;
    const double inv_dx[3] = {1.0 / p->dx[0], 1.0 / p->dx[1], U->ndim == 3 ? 1.0 / p->dx[2] : 0.0};

    cudaStream_t s = ctx->stream;
    const bool params_changed = !U->prepared || U->prep_gamma != p->gamma || U->prep_bc != (int)p->bc ||
                                U->prep_dx[0] != p->dx[0] || U->prep_dx[1] != p->dx[1] ||
                                (U->ndim == 3 && U->prep_dx[2] != p->dx[2]);
    if (params_changed) {
        RIPPLE_CUDA(cudaMemsetAsync(U->ctl->smax, 0, sizeof(U->ctl->smax), s));
        const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
        RIPPLE_CUDA(launch_prep(U->dtype, U->ndim, U->buf[U->cur], U->ctl, g, (int)p->bc, p->gamma, inv_dx,
                                (int)(U->steps_total % 3), grid_for(ctx, total, 256), s));
        U->prepared = true;
        U->prep_gamma = p->gamma;
        U->prep_bc = (int)p->bc;
        for (int d = 0; d < 3; ++d) U->prep_dx[d] = p->dx[d];
    }

    SweepLaunch L{};
    L.sg.f = g;
    L.sg.tiles_x = (g.n[0] + tx - 1) / tx;
    L.sg.tiles_y = (g.n[1] + ty - 1) / ty;
    if (U->ndim == 3) {
        int zc = U->zchunk > 0 ? U->zchunk : 32;
        zc = std::min(zc, g.n[2]);
        L.sg.zchunk = zc;
        L.sg.chunks_z = (g.n[2] + zc - 1) / zc;
    } else {
        L.sg.zchunk = 1;
        L.sg.chunks_z = 1;
    }
    L.sg.items = L.sg.tiles_x * L.sg.tiles_y * L.sg.chunks_z;
    const int occ = std::max(1, sweep_occ(U->dtype, U->ndim, layout, scheme, v));
    L.grid = std::min(L.sg.items, occ * ctx->sm_count);
    L.ctl = U->ctl;
    L.stream = s;
    L.prm.gamma = p->gamma;
    L.prm.cfl = p->cfl;
    for (int d = 0; d < 3; ++d) L.prm.inv_dx[d] = inv_dx[d];
    L.prm.gamma_f = (float)p->gamma;
    L.prm.gm1_f = (float)(p->gamma - 1.0);
    for (int d = 0; d < 3; ++d) L.prm.inv_dx_f[d] = (float)inv_dx[d];
    L.prm.bc = (int)p->bc;

    // one launch per step (unsplit), or one sweep per axis (split: x, then y, then z;
    // each sweep writes the ghost images its successor reads; all read the same dt)
    const int sweeps = split ? U->ndim : 1;
    // the split step of an FP32 field sweeps on strip walks (no tile staging)
    const bool walk = split && U->dtype == RIPPLE_F32 && U->variant < 0;
    WalkLaunch W[3]{};
    if (walk) {
        for (int a = 0; a < U->ndim; ++a) {
            const int wocc = U->ndim == 2 ? force_walk_occ_f32_2d(layout, a) : force_walk_occ_f32_3d(layout, a);
            if (wocc <= 0) return fail(RIPPLE_ERR_INTERNAL, "walk sweep kernel does not fit");
            W[a].wg = walk_geom(g, a, (long long)wocc * ctx->sm_count * kWalkWarps);
            W[a].grid = (int)std::min<long long>((W[a].wg.walks + kWalkWarps - 1) / kWalkWarps,
                                                 (long long)wocc * ctx->sm_count);
            W[a].ctl = U->ctl;
            W[a].stream = s;
            W[a].prm = L.prm;
        }
    }
    for (int64_t n = 0; n < nsteps; ++n) {
        for (int a = 0; a < sweeps; ++a) {
            const int in = U->cur, outb = 1 - U->cur;
            if (walk) {
                W[a].in = U->buf[in];
                W[a].out = U->buf[outb];
                W[a].prm.slot_in = (int)(U->steps_total % 3);
                W[a].prm.first = n == 0;
                W[a].prm.axis = a;
                W[a].prm.last = a == sweeps - 1;
                RIPPLE_CUDA(U->ndim == 2 ? force_walk_launch_f32_2d(layout, a, W[a])
                                         : force_walk_launch_f32_3d(layout, a, W[a]));
                U->cur = outb;
                continue;
            }
            // the row kernel stages AoS planes through the grouped view and
            // stores its results directly (no output map)
            const bool rowk = v == kRowVariant;
            L.map_in = field_map(U, in, rowk && layout == LAYOUT_AOS ? 2 : 0, R, tx, ty, &st);
            if (!L.map_in) return st;
            L.map_out = rowk ? L.map_in : field_map(U, outb, 1, R, tx, ty, &st);
            if (!L.map_out) return st;
            L.out = U->buf[outb];
            L.prm.slot_in = (int)(U->steps_total % 3);
            L.prm.first = n == 0;
            L.prm.axis = split ? a : -1;
            L.prm.last = a == sweeps - 1;
            RIPPLE_CUDA(sweep_launch(U->dtype, U->ndim, layout, scheme, v, L));
            U->cur = outb;
        }
        U->steps_total++;
    }

    if (!stats) return RIPPLE_OK;
    // FP64 compensated totals of the final state
    const int nblocks = 2 * ctx->sm_count;
    const size_t pbytes = (size_t)nblocks * U->ncomp * 2 * sizeof(double);
    if (ctx->partials_bytes < pbytes) {
        RIPPLE_CUDA(cudaStreamSynchronize(s));
        ctx_free(ctx, ctx->partials, ctx->partials_bytes);
        ctx->partials = nullptr;
        ctx->partials_bytes = 0;
        st = ctx_alloc(ctx, pbytes, reinterpret_cast<void**>(&ctx->partials));
        if (st != RIPPLE_OK) return st;
        ctx->partials_bytes = round_up(pbytes, 256);
    }
    RIPPLE_CUDA(launch_totals(U->dtype, U->ncomp, U->buf[U->cur], g, ctx->partials, nblocks, U->ctl, s));
    FieldCtl host{};
    RIPPLE_CUDA(cudaMemcpyAsync(&host, U->ctl, sizeof(FieldCtl), cudaMemcpyDeviceToHost, s));
    RIPPLE_CUDA(cudaStreamSynchronize(s));
    stats->t = nsteps > 0 ? host.t : 0.0;
    stats->dt_last = nsteps > 0 ? host.dt_last : 0.0;
    for (int m = 0; m < 5; ++m) stats->totals[m] = m < U->ncomp ? host.totals[m] : 0.0;
    stats->steps_done = nsteps;
    if (host.err) {
        RIPPLE_CUDA(cudaMemsetAsync(&U->ctl->err, 0, sizeof(unsigned), s));
        RIPPLE_CUDA(cudaMemsetAsync(&U->ctl->counters[4], 0, 4 * sizeof(long long), s));
        return map_dev_err(host.err, &host);
    }
    return RIPPLE_OK;
}

}  // extern "C"
