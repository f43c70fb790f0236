// Internals shared by the C-ABI translation units (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "fsr.h"
#include "fsr_launch.h"

namespace fsri {

constexpr int kNumB = 4;   // B in {2, 4, 8, 16}
inline int b_index(int B) { return B == 2 ? 0 : B == 4 ? 1 : B == 8 ? 2 : B == 16 ? 3 : -1; }

// Method parameters check (error text into h, or the thread's create error when h is NULL).
int check_method(fsr_handle* h, const fsr_params* p);
fsrk::MethodArgs method_args(const fsr_params* p);
fsrk::ImageArgs image_args(const float* img, const uint8_t* mask, float* out, int16_t* seq, int height, int width,
                           int pitch, int iters, int B);
// Batch work tables: [counter u64][first: (n+1) x i64, padded to 16 B]
// [n x ImageArgs, padded to 128 B][n x TileMaps]
size_t table_bytes(int n);
// Fills the host image of a table (images by decreasing K; tile descriptors
// for images whose pitch and alignment allow TMA); returns the total number
// of blocks, or -1 with the error recorded on h.
long long build_table(fsr_handle* h, int n, const fsr_image_desc* d, const fsr_params* p, void* host);
fsrk::BatchArgs batch_args(fsr_handle* h, void* d_table, int n, long long total, const fsr_params* p, int chunk);
// Counter reset + batch kernel on stream s.
cudaError_t launch_batch(const fsrk::BatchArgs& a, const fsr_params* p, fsrk::Schedule sc, int sm_count,
                         cudaStream_t s);
// printf-style error record on a handle (or the thread's create error); returns code.
int fail(fsr_handle* h, int code, const char* fmt, ...);

}  // namespace fsri

struct fsr_handle {
    int device = 0;
    int sm_count = 0;
    char device_name[256] = {0};
    size_t ws_cap = 0;       // 0 = no cap
    size_t ws_used = 0;
    char err[512] = {0};
    std::string cache_path;
    // batch schedules per [precision][B]
    fsrk::Schedule sched[2][fsri::kNumB] = {
        {{fsrk::kWarpsFp32, 1}, {fsrk::kWarpsFp32, 1}, {fsrk::kWarpsFp32, 1}, {fsrk::kWarpsFp32, 1}},
        {{4, 1}, {4, 1}, {4, 1}, {4, 1}}};
    // device staging buffers of fsr_reconstruct_host
    float* d_img = nullptr;
    uint8_t* d_mask = nullptr;
    float* d_out = nullptr;
    size_t stage_pixels = 0;
    // work table of the one-shot batch entry point
    void* d_table = nullptr;
    void* h_table = nullptr;       // pinned host staging of the table
    size_t table_bytes = 0;
    cudaEvent_t table_free = nullptr;
    // device status word of the single-image kernels (fsrk::kStatus* bits)
    unsigned* d_status = nullptr;
    unsigned long long* d_empty = nullptr;   // blocks without a known pixel (inside the status allocation)
    // work counters of FP64 / tensor-core single-image launches, used in turn (self-resetting)
    static constexpr int kWorkSlots = 64;
    unsigned long long* d_work = nullptr;
    unsigned long long work_next = 0;
    // one-image work tables of FP32 single-image launches, used in turn
    static constexpr int kSingleSlots = 64;
    static constexpr size_t kSingleSlotBytes = 512;
    void* h_single = nullptr;   // pinned host images of the slots
    void* d_single = nullptr;
    cudaEvent_t single_ev[kSingleSlots] = {};
    bool single_used[kSingleSlots] = {};
    unsigned long long single_next = 0;
    int inject_tile_fault = 0;     // test hook: next tile-copy launch waits for bytes that never come
};
