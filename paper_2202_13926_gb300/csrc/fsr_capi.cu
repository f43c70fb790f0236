// C-ABI of the GB300 FSR library: handles, argument checks, the batch form
// (work tables, CUDA-graph plans, schedule autotuner) and dispatch to the
// kernels.  Declarations and contracts: include/fsr.h.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "fsr.h"
#include "fsr_internal.h"
#include "fsr_launch.h"

struct fsr_batch {
    fsr_handle* h = nullptr;
    void* d_table = nullptr;
    size_t bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {
thread_local char g_create_err[512] = {0};
}  // namespace

namespace fsri {

int fail(fsr_handle* h, int code, const char* fmt, ...) {
    char* buf = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

int ok(fsr_handle* h) {
    if (h) h->err[0] = 0;
    return FSR_OK;
}

// Keeps the caller's current device across a call.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    cudaError_t set(int dev) {
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        if (prev != dev) {
            e = cudaSetDevice(dev);
            if (e != cudaSuccess) return e;
            changed = true;
        }
        return cudaSuccess;
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    return pa < pb + nb && pb < pa + na;
}

int check_method(fsr_handle* h, const fsr_params* p) {
    if (!p) return fail(h, FSR_ERR_INVALID_ARG, "params is NULL");
    if (p->block <= 0 || p->border < 0) return fail(h, FSR_ERR_INVALID_ARG, "block must be > 0 and border >= 0");
    const int S = p->block + 2 * p->border;
    if (S != fsrk::S && !fsrk::small_supported(S, p->block))
        return fail(h, FSR_ERR_UNSUPPORTED,
                    "support B + 2L = %d with B = %d; this library implements S = 32 (B in {2, 4, 8, 16}), "
                    "S = 24 (B in {4, 8}), S = 16 (B in {2, 4, 8}), S = 8 (B in {2, 4}) and S = 4 (B in {2, 4})",
                    S, p->block);
    if (b_index(p->block) < 0) return fail(h, FSR_ERR_UNSUPPORTED, "block %d not in {2, 4, 8, 16}", p->block);
    if (S != fsrk::S && p->precision != FSR_FP32 && p->precision != FSR_FP64_DEBUG)
        return fail(h, FSR_ERR_UNSUPPORTED, "supports smaller than 32 run FSR_FP32 or FSR_FP64_DEBUG");
    if (!(p->rho > 0.f && p->rho <= 1.f)) return fail(h, FSR_ERR_INVALID_ARG, "rho must be in (0, 1]");
    if (!(p->gamma > 0.f && p->gamma <= 1.f)) return fail(h, FSR_ERR_INVALID_ARG, "gamma must be in (0, 1]");
    if (p->freq_weight != 0 && p->freq_weight != 1) return fail(h, FSR_ERR_INVALID_ARG, "freq_weight must be 0 or 1");
    if (p->precision != FSR_FP32 && p->precision != FSR_FP64_DEBUG && p->precision != FSR_TC_BF16X3 &&
        p->precision != FSR_TC_TF32)
        return fail(h, FSR_ERR_UNSUPPORTED, "precision %d not implemented", p->precision);
    if ((p->precision == FSR_TC_BF16X3 || p->precision == FSR_TC_TF32) && (p->block != 4 || p->iters > 256))
        return fail(h, FSR_ERR_UNSUPPORTED, "tensor-core transform variants are built for B = 4 and K <= 256");
    if (p->update != FSR_UPDATE_SINGLE && p->update != FSR_UPDATE_CONJ_PAIR)
        return fail(h, FSR_ERR_INVALID_ARG, "update must be FSR_UPDATE_SINGLE or FSR_UPDATE_CONJ_PAIR");
    if (p->update == FSR_UPDATE_CONJ_PAIR &&
        (S != fsrk::S || p->block != 4 || (p->precision != FSR_FP32 && p->precision != FSR_FP64_DEBUG)))
        return fail(h, FSR_ERR_UNSUPPORTED, "the conjugate-pair update is built for S = 32, B = 4, FP32 and FP64");
    if (!(p->reuse >= 0.f && p->reuse <= 1.f)) return fail(h, FSR_ERR_INVALID_ARG, "reuse must be in [0, 1]");
    if (p->reuse > 0.f && (S != fsrk::S || p->update != FSR_UPDATE_SINGLE ||
                           (p->precision != FSR_FP32 && p->precision != FSR_FP64_DEBUG)))
        return fail(h, FSR_ERR_UNSUPPORTED,
                    "re-use of reconstructed pixels is built for S = 32, FSR_UPDATE_SINGLE, FP32 and FP64");
    return FSR_OK;
}

int check_image(fsr_handle* h, const float* img, const uint8_t* mask, const float* out, int height, int width,
                int pitch, int iters, bool device_ptrs, int index) {
    if (!img || !mask || !out) return fail(h, FSR_ERR_INVALID_ARG, "image %d: img, mask and out must be non-NULL", index);
    if (height <= 0 || width <= 0)
        return fail(h, FSR_ERR_INVALID_ARG, "image %d: height/width must be > 0 (got %d x %d)", index, height, width);
    if (pitch < width) return fail(h, FSR_ERR_INVALID_ARG, "image %d: pitch (%d) < width (%d)", index, pitch, width);
    if (iters < 0 || iters > 65535) return fail(h, FSR_ERR_INVALID_ARG, "image %d: iters %d out of [0, 65535]", index, iters);
    if (device_ptrs) {
        const size_t n = (size_t)(height - 1) * pitch + width;
        if (ranges_overlap(out, n * sizeof(float), img, n * sizeof(float)) ||
            ranges_overlap(out, n * sizeof(float), mask, n))
            return fail(h, FSR_ERR_INVALID_ARG, "image %d: out overlaps img or mask", index);
    }
    return FSR_OK;
}

fsrk::MethodArgs method_args(const fsr_params* p) {
    fsrk::MethodArgs m;
    m.L = p->border;
    m.rho = p->rho;
    m.gamma = p->gamma;
    m.freq_weight = p->freq_weight;
    return m;
}

fsrk::ImageArgs image_args(const float* img, const uint8_t* mask, float* out, int16_t* seq, int height, int width,
                           int pitch, int iters, int B) {
    fsrk::ImageArgs im;
    im.img = img;
    im.mask = mask;
    im.out = out;
    im.seq = seq;
    im.H = height;
    im.W = width;
    im.pitch = pitch;
    im.nbx = (width + B - 1) / B;
    im.K = iters;
    im.tiles = 0;
    return im;
}

// ---- TMA descriptors of the support tiles (a1) ------------------------------

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library).
EncodeTiled encode_tiled() {
    static const EncodeTiled fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiled>(f);
    }();
    return fn;
}

// Tile copies need 16-byte aligned bases and row strides: img and mask
// 16-byte aligned and the pitch a multiple of 16 elements (16 B of mask).
bool tiles_possible(const float* img, const uint8_t* mask, int pitch) {
    return (reinterpret_cast<uintptr_t>(img) & 15) == 0 && (reinterpret_cast<uintptr_t>(mask) & 15) == 0 &&
           pitch % 16 == 0;
}

// Encodes the image and mask descriptors: [H][W] with row stride pitch,
// boxes of kTileImgCols x S floats and kTileMaskCols x S bytes, zero fill
// outside the image (a pixel outside is unknown).
int encode_tile_maps(fsr_handle* h, const float* img, const uint8_t* mask, int height, int width, int pitch,
                     fsrk::TileMaps* maps) {
    const EncodeTiled enc = encode_tiled();
    if (!enc) return fail(h, FSR_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)height};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint64_t istr[1] = {(cuuint64_t)pitch * sizeof(float)};
    const cuuint32_t ibox[2] = {(cuuint32_t)fsrk::kTileImgCols, (cuuint32_t)fsrk::S};
    CUresult r = enc(&maps->img, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(img), dims, istr, ibox, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, FSR_ERR_CUDA, "cuTensorMapEncodeTiled (image): error %d", (int)r);
    const cuuint64_t mstr[1] = {(cuuint64_t)pitch};
    const cuuint32_t mbox[2] = {(cuuint32_t)fsrk::kTileMaskCols, (cuuint32_t)fsrk::S};
    r = enc(&maps->mask, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(mask), dims, mstr, mbox, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, FSR_ERR_CUDA, "cuTensorMapEncodeTiled (mask): error %d", (int)r);
    return FSR_OK;
}

// Reads and clears the status word (the device must be idle for the handle's
// single-image work); FSR_ERR_TIMEOUT when a kernel's bounded wait gave up.
int read_status(fsr_handle* h) {
    unsigned st = 0;
    cudaError_t e = cudaMemcpy(&st, h->d_status, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "reading the status word: %s", cudaGetErrorString(e));
    if (st == 0) return ok(h);
    if ((e = cudaMemset(h->d_status, 0, sizeof st)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "clearing the status word: %s", cudaGetErrorString(e));
    return fail(h, FSR_ERR_TIMEOUT,
                "status 0x%x: a kernel's bounded wait for a support-tile copy gave up; the warps concerned "
                "stopped and their remaining blocks were not written",
                st);
}

// FP32 single image (and any image of a support smaller than 32): a
// one-image work table in one of the handle's table slots (used in turn; a
// slot is reused once the launch that read it has finished), then the batch
// kernel with the handle's schedule.
int enqueue_single_fp32(fsr_handle* h, const float* img, const uint8_t* mask, int height, int width, int pitch,
                        const fsr_params* p, float* out, cudaStream_t stream) {
    const int slot = (int)(h->single_next++ % fsr_handle::kSingleSlots);
    cudaError_t e;
    if (h->single_used[slot] && (e = cudaEventSynchronize(h->single_ev[slot])) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "waiting for a table slot: %s", cudaGetErrorString(e));
    char* host = static_cast<char*>(h->h_single) + (size_t)slot * fsr_handle::kSingleSlotBytes;
    char* dev = static_cast<char*>(h->d_single) + (size_t)slot * fsr_handle::kSingleSlotBytes;
    fsr_image_desc d;
    d.img = img;
    d.mask = mask;
    d.out = out;
    d.seq_out = p->seq_out;
    d.height = height;
    d.width = width;
    d.pitch = pitch;
    d.iters = p->iters;
    const long long total = build_table(h, 1, &d, p, host);
    if (total < 0) return FSR_ERR_CUDA;
    if ((e = cudaMemcpyAsync(dev, host, table_bytes(1), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
    const fsrk::Schedule sc = h->sched[p->precision == FSR_FP64_DEBUG ? 1 : 0][b_index(p->block)];
    fsrk::BatchArgs a = batch_args(h, dev, 1, total, p, sc.chunk);
    a.empty = h->d_empty;
    a.tx_extra = h->inject_tile_fault ? 16 : 0;
    h->inject_tile_fault = 0;
    const int S = p->block + 2 * p->border;
    if (S != fsrk::S) e = fsrk::launch_batch_small(a, S, p->block, p->precision == FSR_FP64_DEBUG, 1, h->sm_count, stream);
    else if (p->update == FSR_UPDATE_CONJ_PAIR)
        e = fsrk::launch_batch_conj(a, p->precision == FSR_FP64_DEBUG, h->sm_count, stream);
    else e = fsrk::launch_batch_fp32(a, p->block, sc, h->sm_count, stream);
    // the slot is busy until the stream has passed this point (upload and launch)
    const cudaError_t er = cudaEventRecord(h->single_ev[slot], stream);
    if (er == cudaSuccess) h->single_used[slot] = true;
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    if (er != cudaSuccess) return fail(h, FSR_ERR_CUDA, "cudaEventRecord: %s", cudaGetErrorString(er));
    return ok(h);
}

// Re-use form: one launch per wavefront t = a*by + bx (a = ceil(L/B) + 1) of
// the raster order; block (by, bx) of launch t reads the targets of the
// launches before it.  The images of a batch have independent raster orders
// and share the launches: launch t holds wavefront t of every image that has
// one (up to kReuseSegs images per launch; more images take more launches
// for the same t).
int enqueue_reuse_images(fsr_handle* h, int n, const fsrk::ImageArgs* ims, const fsr_params* p,
                         cudaStream_t stream) {
    fsrk::ReuseLaunch a;
    std::memset(&a, 0, sizeof a);
    a.mth = method_args(p);
    a.delta = p->reuse;
    a.slope = (p->border + p->block - 1) / p->block + 1;
    a.empty = h->d_empty;
    long long waves = 0;
    for (int i = 0; i < n; ++i) {
        const long long nby = (ims[i].H + p->block - 1) / p->block;
        waves = std::max(waves, (long long)a.slope * (nby - 1) + ims[i].nbx);
    }
    auto flush = [&](long long t) -> int {
        if (a.nseg == 0) return FSR_OK;
        const cudaError_t e = fsrk::launch_reuse(a, p->block, p->precision == FSR_FP64_DEBUG, h->sm_count, stream);
        a.nseg = 0;
        a.total = 0;
        if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "re-use launch %lld failed: %s", t, cudaGetErrorString(e));
        return FSR_OK;
    };
    for (long long t = 0; t < waves; ++t) {
        a.t = (int)t;
        for (int i = 0; i < n; ++i) {
            // blocks of image i with a*by + bx = t, 0 <= bx < nbx, 0 <= by < nby
            const int nbx = ims[i].nbx, nby = (ims[i].H + p->block - 1) / p->block;
            const long long lo_num = t - (nbx - 1);
            const long long by_lo = lo_num <= 0 ? 0 : (lo_num + a.slope - 1) / a.slope;
            const long long by_hi = std::min<long long>(nby - 1, t / a.slope);
            if (by_hi < by_lo) continue;
            fsrk::ReuseSeg& sg = a.seg[a.nseg++];
            sg.im = ims[i];
            sg.by_lo = (int)by_lo;
            sg.count = (int)(by_hi - by_lo + 1);
            sg.first = a.total;
            a.total += sg.count;
            if (a.nseg == fsrk::kReuseSegs) {
                const int r = flush(t);
                if (r != FSR_OK) return r;
            }
        }
        const int r = flush(t);
        if (r != FSR_OK) return r;
    }
    return ok(h);
}

int enqueue_reuse(fsr_handle* h, const float* img, const uint8_t* mask, int height, int width, int pitch,
                  const fsr_params* p, float* out, cudaStream_t stream) {
    const fsrk::ImageArgs im = image_args(img, mask, out, p->seq_out, height, width, pitch, p->iters, p->block);
    return enqueue_reuse_images(h, 1, &im, p, stream);
}

int enqueue_single(fsr_handle* h, const float* img, const uint8_t* mask, int height, int width, int pitch,
                   const fsr_params* p, float* out, cudaStream_t stream) {
    if (p->reuse > 0.f) return enqueue_reuse(h, img, mask, height, width, pitch, p, out, stream);
    if (p->precision == FSR_FP32 || p->block + 2 * p->border != fsrk::S || p->update == FSR_UPDATE_CONJ_PAIR)
        return enqueue_single_fp32(h, img, mask, height, width, pitch, p, out, stream);
    fsrk::KernelArgs a;
    std::memset(&a, 0, sizeof a);
    a.im = image_args(img, mask, out, p->seq_out, height, width, pitch, p->iters, p->block);
    a.nblocks = (long long)a.im.nbx * ((height + p->block - 1) / p->block);
    a.mth = method_args(p);
    a.status = h->d_status;
    a.empty = h->d_empty;
    a.work = h->d_work + 2 * (h->work_next++ % fsr_handle::kWorkSlots);
    if (tiles_possible(img, mask, pitch)) {
        const int r = encode_tile_maps(h, img, mask, height, width, pitch, &a.maps);
        if (r != FSR_OK) return r;
        a.tiles = 1;
        a.tx_extra = h->inject_tile_fault ? 16 : 0;
        h->inject_tile_fault = 0;
    }
    cudaError_t e;
    if (p->precision == FSR_FP64_DEBUG) e = fsrk::launch_single_fp64(a, p->block, h->sm_count, stream);
    else e = fsrk::launch_single_fp32_tc(a, p->block, p->precision == FSR_TC_BF16X3, h->sm_count, stream);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return ok(h);
}

// ---- batch work tables -----------------------------------------------------
// Layout in one device allocation: [counter u64][first: (n+1) x i64] (padded
// to 16 B) [images: n x ImageArgs] (padded to 128 B) [maps: n x TileMaps].

size_t images_off(int n) {
    return (sizeof(unsigned long long) + sizeof(long long) * (size_t)(n + 1) + 15) & ~(size_t)15;
}

size_t maps_off(int n) { return (images_off(n) + sizeof(fsrk::ImageArgs) * (size_t)n + 127) & ~(size_t)127; }

size_t table_bytes(int n) { return maps_off(n) + sizeof(fsrk::TileMaps) * (size_t)n; }

int check_batch(fsr_handle* h, int n, const fsr_image_desc* d, const fsr_params* p) {
    if (n < 1) return fail(h, FSR_ERR_INVALID_ARG, "batch needs n >= 1 images (got %d)", n);
    if (!d) return fail(h, FSR_ERR_INVALID_ARG, "descs is NULL");
    int r = check_method(h, p);
    if (r != FSR_OK) return r;
    if (p->precision != FSR_FP32 && p->precision != FSR_FP64_DEBUG)
        return fail(h, FSR_ERR_UNSUPPORTED, "the batch form runs FSR_FP32 or FSR_FP64_DEBUG");
    for (int i = 0; i < n; ++i) {
        r = check_image(h, d[i].img, d[i].mask, d[i].out, d[i].height, d[i].width, d[i].pitch, d[i].iters, true, i);
        if (r != FSR_OK) return r;
    }
    return FSR_OK;
}

// Fill the host image of the table; returns the total number of blocks.
long long build_table(fsr_handle* h, int n, const fsr_image_desc* d, const fsr_params* p, void* host) {
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return d[a].iters > d[b].iters; });
    char* base = static_cast<char*>(host);
    auto* counter = reinterpret_cast<unsigned long long*>(base);
    auto* first = reinterpret_cast<long long*>(base + sizeof(unsigned long long));
    auto* imgs = reinterpret_cast<fsrk::ImageArgs*>(base + images_off(n));
    char* maps = base + maps_off(n);
    *counter = 0;
    long long total = 0;
    for (int j = 0; j < n; ++j) {
        const fsr_image_desc& x = d[order[j]];
        imgs[j] = image_args(x.img, x.mask, x.out, x.seq_out, x.height, x.width, x.pitch, x.iters, p->block);
        if (p->block + 2 * p->border == fsrk::S && tiles_possible(x.img, x.mask, x.pitch)) {
            fsrk::TileMaps tm;   // encoded at its own alignment, then copied into the table
            if (encode_tile_maps(h, x.img, x.mask, x.height, x.width, x.pitch, &tm) != FSR_OK) return -1;
            std::memcpy(maps + sizeof(fsrk::TileMaps) * (size_t)j, &tm, sizeof tm);
            imgs[j].tiles = 1;
        }
        first[j] = total;
        total += fsr_num_blocks(x.height, x.width, p->block);
    }
    first[n] = total;
    return total;
}

fsrk::BatchArgs batch_args(fsr_handle* h, void* d_table, int n, long long total, const fsr_params* p, int chunk) {
    char* base = static_cast<char*>(d_table);
    fsrk::BatchArgs a;
    a.counter = reinterpret_cast<unsigned long long*>(base);
    a.first = reinterpret_cast<const long long*>(base + sizeof(unsigned long long));
    a.images = reinterpret_cast<const fsrk::ImageArgs*>(base + images_off(n));
    a.maps = reinterpret_cast<const fsrk::TileMaps*>(base + maps_off(n));
    a.status = h->d_status;
    a.n = n;
    a.total = total;
    a.chunk = chunk;
    a.mth = method_args(p);
    return a;
}

cudaError_t launch_batch(const fsrk::BatchArgs& a, const fsr_params* p, fsrk::Schedule sc, int sm_count,
                         cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int S = p->block + 2 * p->border;
    if (S != fsrk::S)
        return fsrk::launch_batch_small(a, S, p->block, p->precision == FSR_FP64_DEBUG, sc.chunk, sm_count, s);
    if (p->update == FSR_UPDATE_CONJ_PAIR)
        return fsrk::launch_batch_conj(a, p->precision == FSR_FP64_DEBUG, sm_count, s);
    if (a.one_round && p->precision == FSR_FP32) return fsrk::launch_batch_fp32_short(a, p->block, s);
    return (p->precision == FSR_FP64_DEBUG) ? fsrk::launch_batch_fp64(a, p->block, sc, sm_count, s)
                                             : fsrk::launch_batch_fp32(a, p->block, sc, sm_count, s);
}

}  // namespace fsri

namespace {
using namespace fsri;

bool schedule_ok(int precision, int B, const fsrk::Schedule& s) {
    return s.chunk >= 1 && s.chunk <= 64 && fsrk::batch_schedule_supported(precision == FSR_FP64_DEBUG, B, s.warps);
}

void read_schedule_cache(fsr_handle* h) {
    if (h->cache_path.empty()) return;
    FILE* f = fopen(h->cache_path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char name[256];
        int prec, B, warps, chunk;
        if (sscanf(line, "%255[^|]|%d|%d|%d|%d", name, &prec, &B, &warps, &chunk) == 5 &&
            strcmp(name, h->device_name) == 0 && (prec == 0 || prec == 1) && b_index(B) >= 0) {
            fsrk::Schedule s{warps, chunk};
            if (schedule_ok(prec, B, s)) h->sched[prec][b_index(B)] = s;
        }
    }
    fclose(f);
}

void write_schedule_cache(const fsr_handle* h) {
    if (h->cache_path.empty()) return;
    FILE* f = fopen(h->cache_path.c_str(), "w");
    if (!f) return;
    fprintf(f, "# device|precision|B|warps|chunk  (fsr batch schedules)\n");
    const int Bs[kNumB] = {2, 4, 8, 16};
    for (int prec = 0; prec < 2; ++prec)
        for (int i = 0; i < kNumB; ++i)
            fprintf(f, "%s|%d|%d|%d|%d\n", h->device_name, prec, Bs[i], h->sched[prec][i].warps, h->sched[prec][i].chunk);
    fclose(f);
}

int make_plan(fsr_handle* h, int n, const fsr_image_desc* d, const fsr_params* p, fsrk::Schedule sc,
              fsr_batch** out) {
    const size_t bytes = table_bytes(n);
    if (h->ws_cap && h->ws_used + bytes > h->ws_cap)
        return fail(h, FSR_ERR_OOM, "batch table of %zu bytes exceeds the workspace cap of %zu", bytes, h->ws_cap);
    std::vector<char> host(bytes);
    const long long total = build_table(h, n, d, p, host.data());
    if (total < 0) return FSR_ERR_CUDA;
    fsr_batch* b = new (std::nothrow) fsr_batch();
    if (!b) return fail(h, FSR_ERR_OOM, "host allocation of the batch failed");
    b->h = h;
    b->bytes = bytes;
    cudaError_t e = cudaMalloc(&b->d_table, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(h, FSR_ERR_OOM, "cudaMalloc of the batch table (%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    cudaStream_t cs = nullptr;
    if ((e = cudaMemcpy(b->d_table, host.data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
        cudaFree(b->d_table);
        delete b;
        return fail(h, FSR_ERR_CUDA, "batch table upload: %s", cudaGetErrorString(e));
    }
    fsrk::BatchArgs a = batch_args(h, b->d_table, n, total, p, sc.chunk);
    a.empty = h->d_empty;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t el = launch_batch(a, p, sc, h->sm_count, cs);
        e = cudaStreamEndCapture(cs, &b->graph);
        if (el != cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (b->graph) cudaGraphDestroy(b->graph);
        cudaFree(b->d_table);
        delete b;
        return fail(h, FSR_ERR_CUDA, "capturing the batch launch: %s", cudaGetErrorString(e));
    }
    h->ws_used += bytes;
    *out = b;
    return ok(h);
}

void free_plan(fsr_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_table);
    if (b->h) b->h->ws_used -= b->bytes;
    delete b;
}

}  // namespace

extern "C" {

int fsr_create(const fsr_config* cfg, fsr_handle** out) {
    if (!out) return fail(nullptr, FSR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, FSR_ERR_INVALID_ARG, "cfg is NULL");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(nullptr, FSR_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (cfg->device < 0 || cfg->device >= ndev)
        return fail(nullptr, FSR_ERR_INVALID_ARG, "device %d out of range (%d devices)", cfg->device, ndev);
    DeviceGuard g;
    if ((e = g.set(cfg->device)) != cudaSuccess)
        return fail(nullptr, FSR_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, cfg->device)) != cudaSuccess)
        return fail(nullptr, FSR_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(nullptr, FSR_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a only",
                    cfg->device, prop.major, prop.minor);
    if ((e = fsrk::configure_fp32_batch()) != cudaSuccess || (e = fsrk::configure_small()) != cudaSuccess ||
        (e = fsrk::configure_reuse()) != cudaSuccess ||
        (e = fsrk::configure_fp32_sched()) != cudaSuccess || (e = fsrk::configure_fp64()) != cudaSuccess ||
        (e = fsrk::configure_fp64_batch()) != cudaSuccess || (e = fsrk::configure_fp32_tc()) != cudaSuccess ||
        (e = fsrk::configure_conj()) != cudaSuccess || (e = fsrk::configure_fp32_short()) != cudaSuccess)
        return fail(nullptr, FSR_ERR_CUDA, "configuring kernels: %s", cudaGetErrorString(e));
    fsr_handle* h = new (std::nothrow) fsr_handle();
    if (!h) return fail(nullptr, FSR_ERR_OOM, "host allocation of the handle failed");
    if ((e = cudaEventCreateWithFlags(&h->table_free, cudaEventDisableTiming)) != cudaSuccess) {
        delete h;
        return fail(nullptr, FSR_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
    }
    // status word (bytes 0..3), empty-block counter (bytes 8..15), then the
    // work counters of the single-image launches (kWorkSlots x 16 B)
    const size_t sbytes = 16 + 16 * (size_t)fsr_handle::kWorkSlots;
    if ((e = cudaMalloc(&h->d_status, sbytes)) != cudaSuccess ||
        (e = cudaMemset(h->d_status, 0, sbytes)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->d_status);
        cudaEventDestroy(h->table_free);
        delete h;
        return fail(nullptr, FSR_ERR_OOM, "device status word: %s", cudaGetErrorString(e));
    }
    if (table_bytes(1) > fsr_handle::kSingleSlotBytes) {
        cudaFree(h->d_status);
        cudaEventDestroy(h->table_free);
        delete h;
        return fail(nullptr, FSR_ERR_UNSUPPORTED, "internal: one-image table larger than its slot");
    }
    {
        const size_t sb = fsr_handle::kSingleSlotBytes * fsr_handle::kSingleSlots;
        bool okay = cudaMalloc(&h->d_single, sb) == cudaSuccess && cudaMallocHost(&h->h_single, sb) == cudaSuccess;
        for (int i = 0; okay && i < fsr_handle::kSingleSlots; ++i)
            okay = cudaEventCreateWithFlags(&h->single_ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!okay) {
            cudaGetLastError();
            for (cudaEvent_t ev : h->single_ev)
                if (ev) cudaEventDestroy(ev);
            cudaFree(h->d_single);
            if (h->h_single) cudaFreeHost(h->h_single);
            cudaFree(h->d_status);
            cudaEventDestroy(h->table_free);
            delete h;
            return fail(nullptr, FSR_ERR_OOM, "allocating the single-image table slots failed");
        }
    }
    h->d_empty = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(h->d_status) + 8);
    h->d_work = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(h->d_status) + 16);
    h->device = cfg->device;
    h->sm_count = prop.multiProcessorCount;
    snprintf(h->device_name, sizeof h->device_name, "%s", prop.name);
    h->ws_cap = cfg->workspace_bytes;
    if (cfg->schedule_cache) h->cache_path = cfg->schedule_cache;
    read_schedule_cache(h);
    *out = h;
    g_create_err[0] = 0;
    return FSR_OK;
}

int fsr_destroy(fsr_handle* h) {
    if (!h) return FSR_OK;
    {
        DeviceGuard g;
        if (g.set(h->device) == cudaSuccess) {
            cudaFree(h->d_img);
            cudaFree(h->d_mask);
            cudaFree(h->d_out);
            cudaFree(h->d_table);
            cudaFree(h->d_status);
            cudaFree(h->d_single);
            if (h->h_single) cudaFreeHost(h->h_single);
            for (cudaEvent_t ev : h->single_ev)
                if (ev) cudaEventDestroy(ev);
            if (h->h_table) cudaFreeHost(h->h_table);
            if (h->table_free) cudaEventDestroy(h->table_free);
        }
    }
    delete h;
    return FSR_OK;
}

const char* fsr_last_error(const fsr_handle* h) { return h ? h->err : g_create_err; }

long long fsr_num_blocks(int height, int width, int block) {
    if (height <= 0 || width <= 0 || block <= 0) return 0;
    return (long long)((height + block - 1) / block) * ((width + block - 1) / block);
}

int fsr_reconstruct(fsr_handle* h, const float* img, const uint8_t* mask, int height, int width, int pitch,
                    const fsr_params* p, float* out, void* stream) {
    if (!h) return fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    int r = check_method(h, p);
    if (r != FSR_OK) return r;
    r = check_image(h, img, mask, out, height, width, pitch, p->iters, true, 0);
    if (r != FSR_OK) return r;
    DeviceGuard g;
    cudaError_t e = g.set(h->device);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return enqueue_single(h, img, mask, height, width, pitch, p, out, static_cast<cudaStream_t>(stream));
}

int fsr_reconstruct_host(fsr_handle* h, const float* img, const uint8_t* mask, int height, int width, int pitch,
                         const fsr_params* p, float* out, void* stream) {
    if (!h) return fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    int r = check_method(h, p);
    if (r != FSR_OK) return r;
    r = check_image(h, img, mask, out, height, width, pitch, p->iters, false, 0);
    if (r != FSR_OK) return r;
    DeviceGuard g;
    cudaError_t e = g.set(h->device);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    const size_t npix = (size_t)height * width;
    if (npix > h->stage_pixels) {
        const size_t need = npix * (2 * sizeof(float) + 1);
        const size_t have = h->stage_pixels * (2 * sizeof(float) + 1);
        if (h->ws_cap && h->ws_used - have + need > h->ws_cap)
            return fail(h, FSR_ERR_OOM, "staging %zu bytes exceeds the workspace cap of %zu", need, h->ws_cap);
        cudaFree(h->d_img);
        cudaFree(h->d_mask);
        cudaFree(h->d_out);
        h->d_img = nullptr;
        h->d_mask = nullptr;
        h->d_out = nullptr;
        h->ws_used -= have;
        h->stage_pixels = 0;
        if (cudaMalloc(&h->d_img, npix * sizeof(float)) != cudaSuccess || cudaMalloc(&h->d_mask, npix) != cudaSuccess ||
            cudaMalloc(&h->d_out, npix * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h->d_img);
            cudaFree(h->d_mask);
            cudaFree(h->d_out);
            h->d_img = nullptr;
            h->d_mask = nullptr;
            h->d_out = nullptr;
            return fail(h, FSR_ERR_OOM, "cudaMalloc of %zu staging bytes failed", need);
        }
        h->stage_pixels = npix;
        h->ws_used += need;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((e = cudaMemcpy2DAsync(h->d_img, width * sizeof(float), img, (size_t)pitch * sizeof(float),
                               width * sizeof(float), height, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpy2DAsync(h->d_mask, width, mask, (size_t)pitch, width, height, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "host-to-device copy: %s", cudaGetErrorString(e));
    r = enqueue_single(h, h->d_img, h->d_mask, height, width, width, p, h->d_out, s);
    if (r != FSR_OK) return r;
    if ((e = cudaMemcpy2DAsync(out, (size_t)pitch * sizeof(float), h->d_out, width * sizeof(float),
                               width * sizeof(float), height, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "device-to-host copy: %s", cudaGetErrorString(e));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "stream synchronize: %s", cudaGetErrorString(e));
    return read_status(h);
}

int fsr_check_status(fsr_handle* h, void* stream) {
    if (!h) return fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard g;
    cudaError_t e = g.set(h->device);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    if ((e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream))) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "stream synchronize: %s", cudaGetErrorString(e));
    return read_status(h);
}

int fsr_empty_blocks(fsr_handle* h, void* stream, long long* count) {
    if (!h || !count) return fail(h, FSR_ERR_INVALID_ARG, "handle or count is NULL");
    DeviceGuard g;
    cudaError_t e = g.set(h->device);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    unsigned long long c = 0;
    if ((e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream))) != cudaSuccess ||
        (e = cudaMemcpy(&c, h->d_empty, sizeof c, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemset(h->d_empty, 0, sizeof c)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "reading the empty-block counter: %s", cudaGetErrorString(e));
    *count = (long long)c;
    return ok(h);
}

int fsr_inject_tile_wait_fault(fsr_handle* h) {
    if (!h) return fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    h->inject_tile_fault = 1;
    return ok(h);
}

int fsr_reconstruct_batch(fsr_handle* h, int n, const fsr_image_desc* d, const fsr_params* p, void* stream) {
    if (!h) return fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    int r = check_batch(h, n, d, p);
    if (r != FSR_OK) return r;
    DeviceGuard g;
    cudaError_t e = g.set(h->device);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    if (p->reuse > 0.f) {
        // re-use form: every image's wavefront chain, the images sharing the launches
        std::vector<fsrk::ImageArgs> ims((size_t)n);
        for (int i = 0; i < n; ++i)
            ims[i] = image_args(d[i].img, d[i].mask, d[i].out, d[i].seq_out, d[i].height, d[i].width, d[i].pitch,
                                d[i].iters, p->block);
        return enqueue_reuse_images(h, n, ims.data(), p, static_cast<cudaStream_t>(stream));
    }
    // the previous batch of this handle must be done with the table
    if ((e = cudaEventSynchronize(h->table_free)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "waiting for the previous batch: %s", cudaGetErrorString(e));
    const size_t bytes = table_bytes(n);
    if (bytes > h->table_bytes) {
        if (h->ws_cap && h->ws_used - h->table_bytes + bytes > h->ws_cap)
            return fail(h, FSR_ERR_OOM, "batch table of %zu bytes exceeds the workspace cap of %zu", bytes, h->ws_cap);
        cudaFree(h->d_table);
        if (h->h_table) cudaFreeHost(h->h_table);
        h->d_table = nullptr;
        h->h_table = nullptr;
        h->ws_used -= h->table_bytes;
        h->table_bytes = 0;
        if (cudaMalloc(&h->d_table, bytes) != cudaSuccess || cudaMallocHost(&h->h_table, bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h->d_table);
            if (h->h_table) cudaFreeHost(h->h_table);
            h->d_table = nullptr;
            h->h_table = nullptr;
            return fail(h, FSR_ERR_OOM, "allocating the batch table (%zu bytes) failed", bytes);
        }
        h->table_bytes = bytes;
        h->ws_used += bytes;
    }
    const long long total = build_table(h, n, d, p, h->h_table);
    if (total < 0) return FSR_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const fsrk::Schedule sc = h->sched[p->precision][b_index(p->block)];
    if ((e = cudaMemcpyAsync(h->d_table, h->h_table, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "batch table upload: %s", cudaGetErrorString(e));
    fsrk::BatchArgs ba = batch_args(h, h->d_table, n, total, p, sc.chunk);
    ba.empty = h->d_empty;
    if ((e = launch_batch(ba, p, sc, h->sm_count, s)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(e));
    if ((e = cudaEventRecord(h->table_free, s)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
    return ok(h);
}

int fsr_batch_create(fsr_handle* h, int n, const fsr_image_desc* d, const fsr_params* p, fsr_batch** out) {
    if (!h) return fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    if (!out) return fail(h, FSR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int r = check_batch(h, n, d, p);
    if (r != FSR_OK) return r;
    if (p->reuse > 0.f)
        return fail(h, FSR_ERR_UNSUPPORTED, "graph plans run independent blocks (reuse = 0); re-use runs in "
                                            "fsr_reconstruct and fsr_reconstruct_batch");
    DeviceGuard g;
    cudaError_t e = g.set(h->device);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return make_plan(h, n, d, p, h->sched[p->precision][b_index(p->block)], out);
}

int fsr_batch_launch(fsr_batch* b, void* stream) {
    if (!b) return fail(nullptr, FSR_ERR_INVALID_ARG, "batch is NULL");
    DeviceGuard g;
    cudaError_t e = g.set(b->h->device);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(b->h, FSR_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    return ok(b->h);
}

int fsr_batch_destroy(fsr_batch* b) {
    if (!b) return FSR_OK;
    DeviceGuard g;
    g.set(b->h->device);
    free_plan(b);
    return FSR_OK;
}

int fsr_get_schedule(const fsr_handle* h, int block, int precision, fsr_schedule* out) {
    if (!h || !out || b_index(block) < 0 || (precision != FSR_FP32 && precision != FSR_FP64_DEBUG))
        return FSR_ERR_INVALID_ARG;
    const fsrk::Schedule& s = h->sched[precision][b_index(block)];
    out->warps = s.warps;
    out->chunk = s.chunk;
    return FSR_OK;
}

int fsr_set_schedule(fsr_handle* h, int block, int precision, const fsr_schedule* s) {
    if (!h) return fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    if (!s || b_index(block) < 0 || (precision != FSR_FP32 && precision != FSR_FP64_DEBUG))
        return fail(h, FSR_ERR_INVALID_ARG, "bad block, precision or schedule pointer");
    const fsrk::Schedule sc{s->warps, s->chunk};
    if (!schedule_ok(precision, block, sc))
        return fail(h, FSR_ERR_UNSUPPORTED, "schedule warps=%d chunk=%d is not instantiated for B=%d", s->warps,
                    s->chunk, block);
    h->sched[precision][b_index(block)] = sc;
    return ok(h);
}

int fsr_autotune_batch(fsr_handle* h, int n, const fsr_image_desc* d, const fsr_params* p, fsr_schedule* best,
                       float* best_ms) {
    if (!h) return fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    int r = check_batch(h, n, d, p);
    if (r != FSR_OK) return r;
    if (p->reuse > 0.f)
        return fail(h, FSR_ERR_UNSUPPORTED, "the schedule autotuner times independent blocks (reuse = 0)");
    DeviceGuard g;
    cudaError_t e = g.set(h->device);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    cudaStream_t s = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "autotune setup: %s", cudaGetErrorString(e));
    const int warps_c[3] = {fsrk::kWarpsFp32, 12, 16};
    const int chunk_c[4] = {1, 2, 4, 8};
    fsrk::Schedule win = h->sched[p->precision][b_index(p->block)];
    float win_ms = -1.f;
    int rc = FSR_OK;
    for (int wi = 0; wi < 3 && rc == FSR_OK; ++wi) {
        for (int ci = 0; ci < 4 && rc == FSR_OK; ++ci) {
            const fsrk::Schedule sc{warps_c[wi], chunk_c[ci]};
            if (!schedule_ok(p->precision, p->block, sc)) continue;
            fsr_batch* plan = nullptr;
            rc = make_plan(h, n, d, p, sc, &plan);
            if (rc != FSR_OK) break;
            float ms = 0.f;
            // one warm-up launch, then the mean of two timed launches
            e = cudaGraphLaunch(plan->exec, s);
            if (e == cudaSuccess) e = cudaEventRecord(t0, s);
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = cudaGraphLaunch(plan->exec, s);
            if (e == cudaSuccess) e = cudaEventRecord(t1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            free_plan(plan);
            if (e != cudaSuccess) {
                rc = fail(h, FSR_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(e));
                break;
            }
            ms *= 0.5f;
            if (win_ms < 0.f || ms < win_ms) {
                win_ms = ms;
                win = sc;
            }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaStreamDestroy(s);
    if (rc != FSR_OK) return rc;
    h->sched[p->precision][b_index(p->block)] = win;
    write_schedule_cache(h);
    if (best) {
        best->warps = win.warps;
        best->chunk = win.chunk;
    }
    if (best_ms) *best_ms = win_ms;
    return ok(h);
}

}  // extern "C"
