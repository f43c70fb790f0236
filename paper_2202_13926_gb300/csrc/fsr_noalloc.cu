// Batch reconstruction that never allocates device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework
// which owns the whole device-memory budget through its own allocator,
// real-time loops where an allocation (which may synchronise the device and
// stall every stream) is not acceptable, and plug-ins that are not allowed to
// keep device memory of their own between calls.  For them the work table of
// the batch kernel (its scratch memory: the work counter, the block prefix
// sums and the per-image arguments) lives in a fixed array in the module's
// own static device memory instead of a buffer from the allocator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>

#include "fsr.h"
#include "fsr_launch.h"

namespace {

constexpr size_t kScratchBytes = FSR_STATIC_SCRATCH_BYTES;
constexpr int kMaxImages = FSR_STATIC_MAX_IMAGES;
constexpr int kMaxDevices = 64;

// The scratch of every call on a device.  In host code this name is only a
// stand-in; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_batch_scratch[kScratchBytes];

struct DeviceSetup {
    bool done = false;
    void* scratch = nullptr;   // device address of g_batch_scratch on this device
    int sm_count = 0;
};

std::mutex g_mu;                                      // guards g_setup
DeviceSetup g_setup[kMaxDevices];

// The table of one call travels to the device in the launch parameters of a
// small kernel that copies it into g_batch_scratch: nothing in host memory is
// read after the call returns, and no host buffer is shared between calls.
struct TableImage {
    int bytes;                                        // used bytes, a multiple of 16
    alignas(16) unsigned char data[kScratchBytes];
};

__global__ void put_table(const __grid_constant__ TableImage t) {
    for (int i = 16 * (int)threadIdx.x; i < t.bytes; i += 16 * (int)blockDim.x)
        *reinterpret_cast<uint4*>(g_batch_scratch + i) = *reinterpret_cast<const uint4*>(t.data + i);
}

int report(char* err, size_t err_len, int code, const char* fmt, ...) {
    if (err && err_len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, err_len, fmt, ap);
        va_end(ap);
    }
    return code;
}

// Table layout: [counter u64][first: (n+1) x i64, padded to 16 B][n x ImageArgs]
size_t images_offset(int n) {
    return (sizeof(unsigned long long) + sizeof(long long) * (size_t)(n + 1) + 15) & ~(size_t)15;
}

}  // namespace

extern "C" int fsr_reconstruct_batch_static(int n, const fsr_image_desc* d, const fsr_params* p, void* stream,
                                            char* err, size_t err_len) {
    if (err && err_len) err[0] = 0;
    if (n < 1 || !d || !p) return report(err, err_len, FSR_ERR_INVALID_ARG, "need n >= 1, descs and params");
    const size_t bytes = images_offset(n) + sizeof(fsrk::ImageArgs) * (size_t)n;
    if (n > kMaxImages || bytes > kScratchBytes)
        return report(err, err_len, FSR_ERR_INVALID_ARG,
                      "%d images exceed the static scratch of this entry point (at most %d images, %zu bytes); "
                      "split the batch or use fsr_reconstruct_batch",
                      n, kMaxImages, kScratchBytes);
    if (p->block + 2 * p->border != fsrk::S || !(p->block == 2 || p->block == 4 || p->block == 8 || p->block == 16))
        return report(err, err_len, FSR_ERR_UNSUPPORTED, "block %d / border %d: the allocation-free entry point implements S = 32, B in {2,4,8,16}",
                      p->block, p->border);
    if (!(p->rho > 0.f && p->rho <= 1.f) || !(p->gamma > 0.f && p->gamma <= 1.f) ||
        (p->freq_weight != 0 && p->freq_weight != 1))
        return report(err, err_len, FSR_ERR_INVALID_ARG, "rho and gamma must be in (0, 1], freq_weight 0 or 1");
    if (p->precision != FSR_FP32 && p->precision != FSR_FP64_DEBUG)
        return report(err, err_len, FSR_ERR_UNSUPPORTED, "precision %d not implemented", p->precision);
    if (p->update != FSR_UPDATE_SINGLE)
        return report(err, err_len, FSR_ERR_UNSUPPORTED, "the allocation-free entry point runs FSR_UPDATE_SINGLE only");
    if (p->reuse != 0.f)
        return report(err, err_len, FSR_ERR_UNSUPPORTED, "the allocation-free entry point runs independent blocks (reuse = 0)");
    for (int i = 0; i < n; ++i) {
        const fsr_image_desc& x = d[i];
        if (!x.img || !x.mask || !x.out || x.height <= 0 || x.width <= 0 || x.pitch < x.width || x.iters < 0 ||
            x.iters > 65535)
            return report(err, err_len, FSR_ERR_INVALID_ARG, "image %d: bad pointers, geometry or iters", i);
        const size_t np = (size_t)(x.height - 1) * x.pitch + x.width;
        const char* o = reinterpret_cast<const char*>(x.out);
        const char* a = reinterpret_cast<const char*>(x.img);
        const char* m = reinterpret_cast<const char*>(x.mask);
        if ((o < a + np * sizeof(float) && a < o + np * sizeof(float)) || (o < m + np && m < o + np * sizeof(float)))
            return report(err, err_len, FSR_ERR_INVALID_ARG, "image %d: out overlaps img or mask", i);
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report(err, err_len, FSR_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return report(err, err_len, FSR_ERR_UNSUPPORTED, "device %d exceeds the %d devices this entry point tracks",
                      dev, kMaxDevices);

    std::unique_lock<std::mutex> lock(g_mu);
    DeviceSetup& su = g_setup[dev];
    if (!su.done) {
        // once per device, with that device current
        cudaDeviceProp prop;
        if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess)
            return report(err, err_len, FSR_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
        if (!(prop.major == 10 && prop.minor == 3))
            return report(err, err_len, FSR_ERR_UNSUPPORTED, "device %d is sm_%d%d; built for sm_103a only", dev,
                          prop.major, prop.minor);
        void* ptr = nullptr;
        if ((e = cudaGetSymbolAddress(&ptr, g_batch_scratch)) != cudaSuccess)
            return report(err, err_len, FSR_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        if ((e = fsrk::configure_fp32_batch()) != cudaSuccess || (e = fsrk::configure_fp64_batch()) != cudaSuccess)
            return report(err, err_len, FSR_ERR_CUDA, "configuring kernels: %s", cudaGetErrorString(e));
        su.scratch = ptr;
        su.sm_count = prop.multiProcessorCount;
        su.done = true;
    }
    void* const scratch = su.scratch;
    const int sm_count = su.sm_count;
    lock.unlock();

    // The table: images by decreasing K, prefix sums of their block counts,
    // and a zero work counter (the array keeps the last call's contents, so
    // the counter is cleared by this copy).
    TableImage tab;
    tab.bytes = (int)((bytes + 15) & ~(size_t)15);
    std::memset(tab.data, 0, (size_t)tab.bytes);
    int order[kMaxImages];
    std::iota(order, order + n, 0);
    std::stable_sort(order, order + n, [&](int a, int b) { return d[a].iters > d[b].iters; });
    auto* first = reinterpret_cast<long long*>(tab.data + sizeof(unsigned long long));
    auto* imgs = reinterpret_cast<fsrk::ImageArgs*>(tab.data + images_offset(n));
    long long total = 0;
    for (int j = 0; j < n; ++j) {
        const fsr_image_desc& x = d[order[j]];
        fsrk::ImageArgs& im = imgs[j];
        im.img = x.img;
        im.mask = x.mask;
        im.out = x.out;
        im.seq = x.seq_out;
        im.H = x.height;
        im.W = x.width;
        im.pitch = x.pitch;
        im.nbx = (x.width + p->block - 1) / p->block;
        im.K = x.iters;
        first[j] = total;
        total += (long long)((x.height + p->block - 1) / p->block) * im.nbx;
    }
    first[n] = total;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    put_table<<<1, 128, 0, s>>>(tab);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return report(err, err_len, FSR_ERR_CUDA, "table copy: %s", cudaGetErrorString(e));

    fsrk::BatchArgs ba;
    unsigned char* base = static_cast<unsigned char*>(scratch);
    ba.counter = reinterpret_cast<unsigned long long*>(base);
    ba.first = reinterpret_cast<const long long*>(base + sizeof(unsigned long long));
    ba.images = reinterpret_cast<const fsrk::ImageArgs*>(base + images_offset(n));
    ba.n = n;
    ba.total = total;
    ba.chunk = 1;
    ba.mth.L = p->border;
    ba.mth.rho = p->rho;
    ba.mth.gamma = p->gamma;
    ba.mth.freq_weight = p->freq_weight;
    const fsrk::Schedule sc{p->precision == FSR_FP64_DEBUG ? 4 : fsrk::kWarpsFp32, 1};
    e = (p->precision == FSR_FP64_DEBUG) ? fsrk::launch_batch_fp64(ba, p->block, sc, sm_count, s)
                                         : fsrk::launch_batch_fp32(ba, p->block, sc, sm_count, s);
    if (e != cudaSuccess) return report(err, err_len, FSR_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(e));
    return FSR_OK;
}
