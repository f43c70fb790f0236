// C-ABI of the GB300 FSR library: handle management, argument checks and
// dispatch to the per-block kernels.  Declarations and contracts: include/fsr.h.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "fsr.h"
#include "fsr_launch.h"

struct fsr_handle {
    int device = 0;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    size_t ws_cap = 0;       // 0 = no cap
    size_t ws_used = 0;
    char err[512] = {0};
    // device staging buffers of fsr_reconstruct_host
    float* d_img = nullptr;
    uint8_t* d_mask = nullptr;
    float* d_out = nullptr;
    size_t stage_pixels = 0;
};

namespace {

thread_local char g_create_err[512] = {0};

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

int check_params(fsr_handle* h, int height, int width, int pitch, const fsr_params* p) {
    if (!p) return fail(h, FSR_ERR_INVALID_ARG, "params is NULL");
    if (height <= 0 || width <= 0) return fail(h, FSR_ERR_INVALID_ARG, "height/width must be > 0 (got %d x %d)", height, width);
    if (pitch < width) return fail(h, FSR_ERR_INVALID_ARG, "pitch (%d) < width (%d)", pitch, width);
    if (p->block <= 0 || p->border < 0) return fail(h, FSR_ERR_INVALID_ARG, "block must be > 0 and border >= 0");
    if (p->block + 2 * p->border != fsrk::S)
        return fail(h, FSR_ERR_UNSUPPORTED, "support B + 2L = %d; this build implements S = 32", p->block + 2 * p->border);
    if (p->block != 2 && p->block != 4 && p->block != 8 && p->block != 16)
        return fail(h, FSR_ERR_UNSUPPORTED, "block %d not in {2, 4, 8, 16}", p->block);
    if (p->iters < 0 || p->iters > 65535) return fail(h, FSR_ERR_INVALID_ARG, "iters %d out of [0, 65535]", p->iters);
    if (!(p->rho > 0.f && p->rho <= 1.f)) return fail(h, FSR_ERR_INVALID_ARG, "rho must be in (0, 1]");
    if (!(p->gamma > 0.f && p->gamma <= 1.f)) return fail(h, FSR_ERR_INVALID_ARG, "gamma must be in (0, 1]");
    if (p->freq_weight != 0 && p->freq_weight != 1) return fail(h, FSR_ERR_INVALID_ARG, "freq_weight must be 0 or 1");
    if (p->precision != FSR_FP32 && p->precision != FSR_FP64_DEBUG)
        return fail(h, FSR_ERR_UNSUPPORTED, "precision %d not implemented", p->precision);
    return FSR_OK;
}

int enqueue(fsr_handle* h, const float* img, const uint8_t* mask, int height, int width,
            int pitch, const fsr_params* p, float* out, cudaStream_t stream) {
    fsrk::KernelArgs a;
    a.img = img;
    a.mask = mask;
    a.out = out;
    a.seq = p->seq_out;
    a.H = height;
    a.W = width;
    a.pitch = pitch;
    a.nbx = (width + p->block - 1) / p->block;
    a.nblocks = (long long)a.nbx * ((height + p->block - 1) / p->block);
    a.L = p->border;
    a.K = p->iters;
    a.rho = p->rho;
    a.gamma = p->gamma;
    a.freq_weight = p->freq_weight;
    cudaError_t e = (p->precision == FSR_FP64_DEBUG)
                        ? fsrk::launch_fp64(a, p->block, h->sm_count, stream)
                        : fsrk::launch_fp32(a, p->block, h->sm_count, stream);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return ok(h);
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
    if ((e = fsrk::configure_fp32()) != cudaSuccess || (e = fsrk::configure_fp64()) != cudaSuccess)
        return fail(nullptr, FSR_ERR_CUDA, "configuring kernels: %s", cudaGetErrorString(e));
    fsr_handle* h = new (std::nothrow) fsr_handle();
    if (!h) return fail(nullptr, FSR_ERR_OOM, "host allocation of the handle failed");
    h->device = cfg->device;
    h->sm_count = prop.multiProcessorCount;
    h->cc_major = prop.major;
    h->cc_minor = prop.minor;
    h->ws_cap = cfg->workspace_bytes;
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

int fsr_reconstruct(fsr_handle* h, const float* img, const uint8_t* mask, int height, int width,
                    int pitch, const fsr_params* p, float* out, void* stream) {
    if (!h) return fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    if (!img || !mask || !out) return fail(h, FSR_ERR_INVALID_ARG, "img, mask and out must be non-NULL");
    int r = check_params(h, height, width, pitch, p);
    if (r != FSR_OK) return r;
    const size_t n = (size_t)(height - 1) * pitch + width;
    if (ranges_overlap(out, n * sizeof(float), img, n * sizeof(float)) ||
        ranges_overlap(out, n * sizeof(float), mask, n))
        return fail(h, FSR_ERR_INVALID_ARG, "out overlaps img or mask");
    DeviceGuard g;
    cudaError_t e = g.set(h->device);
    if (e != cudaSuccess) return fail(h, FSR_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return enqueue(h, img, mask, height, width, pitch, p, out, static_cast<cudaStream_t>(stream));
}

int fsr_reconstruct_host(fsr_handle* h, const float* img, const uint8_t* mask, int height, int width,
                         int pitch, const fsr_params* p, float* out, void* stream) {
    if (!h) return fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    if (!img || !mask || !out) return fail(h, FSR_ERR_INVALID_ARG, "img, mask and out must be non-NULL");
    int r = check_params(h, height, width, pitch, p);
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
        cudaFree(h->d_img); cudaFree(h->d_mask); cudaFree(h->d_out);
        h->d_img = nullptr; h->d_mask = nullptr; h->d_out = nullptr;
        h->ws_used -= have;
        h->stage_pixels = 0;
        if (cudaMalloc(&h->d_img, npix * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&h->d_mask, npix) != cudaSuccess ||
            cudaMalloc(&h->d_out, npix * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h->d_img); cudaFree(h->d_mask); cudaFree(h->d_out);
            h->d_img = nullptr; h->d_mask = nullptr; h->d_out = nullptr;
            return fail(h, FSR_ERR_OOM, "cudaMalloc of %zu staging bytes failed", need);
        }
        h->stage_pixels = npix;
        h->ws_used += need;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((e = cudaMemcpy2DAsync(h->d_img, width * sizeof(float), img, (size_t)pitch * sizeof(float),
                               width * sizeof(float), height, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpy2DAsync(h->d_mask, width, mask, (size_t)pitch, width, height,
                               cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "host-to-device copy: %s", cudaGetErrorString(e));
    r = enqueue(h, h->d_img, h->d_mask, height, width, width, p, h->d_out, s);
    if (r != FSR_OK) return r;
    if ((e = cudaMemcpy2DAsync(out, (size_t)pitch * sizeof(float), h->d_out, width * sizeof(float),
                               width * sizeof(float), height, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "device-to-host copy: %s", cudaGetErrorString(e));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(h, FSR_ERR_CUDA, "stream synchronize: %s", cudaGetErrorString(e));
    return ok(h);
}

}  // extern "C"
