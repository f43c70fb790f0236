// Per-block FSR on sm_103a: one warp owns one 32 x 32 support block.
//
// Sec. II / Sec. III of Regensky et al. (MMSP 2020), re-laid out for GB300:
//   * lane n first holds column n of the support, then (after one transpose
//     through shared memory) lane k holds row k of the spectrum: R_w[k][0..31]
//     lives in 64 registers of lane k for the whole iteration;
//   * the forward transform is one complex 32 x 32 DFT of z = x + j 2^e w
//     (x = (f~ - mu) w, the weighted signal of Eq. 7 less its weighted mean
//     mu, and w of Eq. 5), done as two register-resident radix-2 FFT passes;
//     Q = F2{x} and W are separated with the conjugate-symmetry identities,
//     which makes both exactly Hermitian.  R_w = mu W + Q exactly; while only
//     the DC basis image is selected, R_w is kept as a W + Q with the scalar
//     a absorbing every DC update (no rounding of the spectrum); at the first
//     other selection a W is folded into Q (this keeps the FP32 spectrum
//     within a few ulps of the FP64 one while the DC term dominates);
//   * W is kept in shared memory; an FP32 row holds W[i][0..31] followed by
//     W[i][0..15] (48 entries), so the circularly shifted row
//     W[(k-u) mod S][(l-v) mod S], l = 0..31 of Eqs. (12), (14), (15) is read
//     as two runs of 16 consecutive entries starting at columns s and
//     (s + 16) mod S, s = (S - v) mod S: no index wrap inside a run;
//   * the support tile of image and mask comes in by two TMA tile copies per
//     block (image pitch permitting); pixels outside the image arrive as the
//     copy's zero fill, i.e. as unknown;
//   * argmax (Eq. 8): each lane keeps the running maximum of its row, one
//     warp max-reduction gives the maximum M, the lowest lane whose row holds
//     M is u, that lane publishes its row, and the lowest column with
//     objective M is v.  The objective is recomputed with the same rounded
//     operations, so the equality tests are exact and the tie rule (lowest
//     k*S + l) is kept bit for bit;
//   * the inverse transform is only needed at the B x B target pixels: every
//     iteration adds Re(gamma p e^{+j2pi(um+vn)/S}) to those pixels, which
//     equals Re IDFT2(G) with G of Eq. (11) (the S^2 of Eq. 11 cancels the
//     1/S^2 of the inverse).
#pragma once

#include <cstdint>
#include <cuda.h>          // CUtensorMap (type only)
#include <cuda_runtime.h>

namespace fsrk {

constexpr int S = 32;                 // support size of this kernel family
constexpr int TSTRIDE = S + 1;        // transpose buffer row stride
constexpr unsigned FULL = 0xffffffffu;

// One image of a launch: device pointers (caller-owned) and geometry.
struct ImageArgs {
    const float* img;
    const uint8_t* mask;
    float* out;
    int16_t* seq;        // optional: N*K selected indices of this image
    int H, W, pitch;     // geometry (pitch in elements, shared by img, mask, out)
    int nbx;             // ceil(W / B): blocks per block row
    int K;               // iterations of this image
    int tiles;           // batch form: 1 = maps[image] holds this image's tile descriptors
};

// Parameters shared by every image of a launch.
struct MethodArgs {
    int L;               // border
    float rho, gamma;
    int freq_weight;
};

// TMA descriptors of one image: the support tile of every block is one 2-D
// tile copy of the image (kTileImgCols x 32 floats) and one of the mask
// (kTileMaskCols x 32 bytes); coordinates are rounded down to 16-byte
// boundaries and the lane offset is taken in shared memory.
constexpr int kTileImgCols = S + 4;     // 144 B rows: x rounded down to a multiple of 4 floats
constexpr int kTileMaskCols = S + 16;   // 48 B rows: x rounded down to a multiple of 16 bytes
constexpr unsigned kTileImgBytes = 4u * kTileImgCols * S;   // 4608
constexpr unsigned kTileMaskBytes = 1u * kTileMaskCols * S; // 1536
constexpr unsigned kTileBytes = kTileImgBytes + kTileMaskBytes;
struct TileMaps {
    CUtensorMap img;    // FLOAT32 [H][W], row stride pitch * 4 B, box {kTileImgCols, S}
    CUtensorMap mask;   // UINT8   [H][W], row stride pitch B,     box {kTileMaskCols, S}
};

// Device status word bits (set by kernels, read and cleared by the host).
constexpr unsigned kStatusTileWait = 1u;   // a bounded wait on a tile copy gave up

// Single image: warps take blocks one at a time from a device work counter.
struct KernelArgs {
    ImageArgs im;
    long long nblocks;   // N
    unsigned long long* work;   // [next block, finished warps]: zero at launch; the last warp resets both
    MethodArgs mth;
    unsigned* status;    // device status word (kStatus* bits)
    unsigned long long* empty;   // optional: += blocks without a known pixel
    int tiles;           // 1: support tiles by TMA through `maps`; 0: plain loads
    int tx_extra;        // test hook: extra bytes each tile wait expects (0 in use)
    TileMaps maps;
};

// Many images, dynamic schedule: warps take chunks of the concatenated block
// list (images ordered by decreasing K) from a device counter.
struct TileMaps;
struct BatchArgs {
    const ImageArgs* images;     // n images, device memory
    const long long* first;      // n + 1 prefix sums of the block counts
    int n;
    long long total;             // first[n]
    unsigned long long* counter; // zero at launch
    int chunk;                   // blocks taken per counter increment
    MethodArgs mth;
    unsigned long long* empty = nullptr;   // optional: += blocks without a known pixel
    const TileMaps* maps = nullptr;        // optional: n tile descriptors (device, 64-byte aligned)
    unsigned* status = nullptr;            // device status word (needed with maps)
    int tx_extra = 0;                      // test hook of the tile wait (0 in use)
    int one_round = 0;                     // 1: run the ONE_ROUND form of the FP32 S = 32 batch kernel
                                           // (a warp takes one chunk, then its CTA ends)
};

// cos(pi t / 16) for t = 0..8 (mathematical constants).
__host__ __device__ constexpr double cos_pi16_base(int t) {
    return t == 0 ? 1.0
         : t == 1 ? 0.980785280403230449126182236134239037
         : t == 2 ? 0.923879532511286756128183189396788287
         : t == 3 ? 0.831469612302545237078788377617905757
         : t == 4 ? 0.707106781186547524400844362104849039
         : t == 5 ? 0.555570233019602224742830813948532874
         : t == 6 ? 0.382683432365089771728459984030398867
         : t == 7 ? 0.195090322016128267848284868477022241
         : 0.0;
}
// cos(2 pi t / 32) and sin(2 pi t / 32) for any integer t, exact on the axes.
__host__ __device__ constexpr double cos_2pi32(int t) {
    t &= 31;
    return t <= 8 ? cos_pi16_base(t)
         : t <= 16 ? -cos_pi16_base(16 - t)
         : t <= 24 ? -cos_pi16_base(t - 16)
         : cos_pi16_base(32 - t);
}
__host__ __device__ constexpr double sin_2pi32(int t) { return cos_2pi32(t - 8); }

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

__host__ __device__ constexpr int brev5(int i) {
    return ((i & 1) << 4) | ((i & 2) << 2) | (i & 4) | ((i & 8) >> 2) | ((i & 16) >> 4);
}

// Explicitly rounded operations: the objective must be bit-reproducible.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// obj = w_f (Re^2 + Im^2) (Eq. 8 / the objective of Sec. III-B).
template <typename T>
__device__ __forceinline__ T objective(T re, T im, T wf) {
    return mul_rn(wf, fma_rn(im, im, mul_rn(re, re)));
}

// In-register radix-2 decimation-in-time FFT of length 32, natural order in
// and out, X[k] = sum_m x[m] e^{-j 2 pi k m / 32}.  Twiddles are compile-time
// constants; the multiplications by 1 and -j are skipped.
template <typename T>
__device__ __forceinline__ void fft32(T (&re)[32], T (&im)[32]) {
    T ar[32], ai[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        ar[i] = re[brev5(i)];
        ai[i] = im[brev5(i)];
    }
#pragma unroll
    for (int half = 1; half < 32; half *= 2) {
#pragma unroll
        for (int j = 0; j < 32; j += 2 * half) {
#pragma unroll
            for (int t = 0; t < half; ++t) {
                const int tw = t * (16 / half);  // e^{-j 2 pi tw / 32}
                const T br = ar[j + t + half], bi = ai[j + t + half];
                T xr, xi;
                if (tw == 0) {
                    xr = br; xi = bi;
                } else if (tw == 8) {  // times -j
                    xr = bi; xi = -br;
                } else {
                    const T c = T(cos_2pi32(tw)), s = T(-sin_2pi32(tw));
                    xr = br * c - bi * s;
                    xi = br * s + bi * c;
                }
                ar[j + t + half] = ar[j + t] - xr;
                ai[j + t + half] = ai[j + t] - xi;
                ar[j + t] = ar[j + t] + xr;
                ai[j + t] = ai[j + t] + xi;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        re[i] = ar[i];
        im[i] = ai[i];
    }
}

__device__ __forceinline__ float max3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ float warp_max(float x) {
    // objective values are >= +0, so their bit patterns order like the values
    return __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(x)));
}
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(FULL, x, o));
    return x;
}

// Arithmetic of the 2-D DFTs: SIMT FFTs, or (precision study) GEMMs on the
// tensor cores with TF32 operands or BF16 hi/lo split products (the
// tcgen05 transform of fsr_tc5.cuh).
enum class Dft { SIMT = 0, TF32 = 1, BF16X3 = 2 };

// The transform context of the SIMT path (no tensor-core state).
struct NoTc {
    __device__ void dft2(float (&)[32], float (&)[32], int) {}
};

// Row stride (in complex elements) of the stored W rows, chosen so that 32
// lanes reading 32 different rows at one column hit distinct banks (128-bit
// loads).  FP64 rows hold 64 entries (the row twice); FP32 rows hold 48
// (the row and its first half again): every 16 consecutive entries of the
// circular row are contiguous, which is what the FP32 loop reads.
template <typename T> struct WRow;
template <> struct WRow<float> { static constexpr int stride = S + S / 2 + 2; };  // 48 entries + pad: 400 B
template <> struct WRow<double> { static constexpr int stride = 2 * S + 1; };  // 1040 B

// Row stride of the w_f table: one pad entry, so that 32 lanes reading
// w_f[lane][l] hit 32 different banks.
constexpr int WFS = S + 1;

template <typename T>
struct SmemLayout {
    using T2 = typename Vec2<T>::type;
    static constexpr int WS = WRow<T>::stride;
    // CTA-shared tables
    static constexpr size_t w0_off = 0;                                 // S*S T
    static constexpr size_t wf_off = w0_off + sizeof(T) * S * S;        // S*WFS T
    static constexpr size_t cs_off = wf_off + sizeof(T) * S * WFS;      // S T2
    static constexpr size_t warp0_off = cs_off + sizeof(T2) * S;
    // per warp: W rows, then the published row
    static constexpr size_t w_elems = (size_t)S * WS;
    static constexpr size_t per_warp = sizeof(T2) * (w_elems + S);
    // after the warps' areas: one tile-copy mbarrier (8 B) per warp, then the
    // parity (4 B) of the phase each warp waits for next
    static constexpr size_t bar_off(int warps) { return warp0_off + per_warp * (size_t)warps; }
    static constexpr size_t parity_off(int warps) { return bar_off(warps) + 8 * (size_t)warps; }
    static constexpr size_t bytes(int warps) { return bar_off(warps) + ((12 * (size_t)warps + 127) & ~(size_t)127); }
    // the support tile lands in the warp's W area before that area is used;
    // 128-byte offsets keep both tile copies' destinations aligned
    static_assert(kTileBytes <= sizeof(T2) * w_elems, "support tile must fit the W area");
    static_assert(warp0_off % 128 == 0 && per_warp % 128 == 0, "warp areas must be 128-byte aligned");
};

// Number of target pixels each lane accumulates for a B x B target.
template <int B> struct TargetPix { static constexpr int P = (B * B + 31) / 32; };

// Per-block values shared by the phases.
template <typename T>
struct BlockState {
    T W0;   // W[0][0] = sum of w
    T mu;   // weighted mean of the known values: R_w = mu W + Q at the start
};

// ---- a1 by TMA: one tile copy of image and mask per block ----------------
// The wait on a copy is bounded: after kTileWaitPolls polls of at most
// kTileWaitHintNs each (about a second) the warp records kStatusTileWait in
// the status word and stops taking blocks; the host reports FSR_ERR_TIMEOUT.
constexpr int kTileWaitPolls = 1 << 16;
constexpr unsigned kTileWaitHintNs = 20000;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tile_bar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Lane 0: expect `bytes` on `bar` and start both copies of the support whose
// top-left pixel is (y0, x0).
__device__ __forceinline__ void tile_issue(const TileMaps* maps, uint32_t dst, uint32_t bar, int y0, int x0,
                                           unsigned bytes) {
    const uint64_t mi = reinterpret_cast<uint64_t>(&maps->img);
    const uint64_t mm = reinterpret_cast<uint64_t>(&maps->mask);
    // the W area was last written and read through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(mi), "r"(x0 & ~3), "r"(y0), "r"(bar)
        : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst + kTileImgBytes), "l"(mm), "r"(x0 & ~15), "r"(y0), "r"(bar)
        : "memory");
}

// Every lane: wait (bounded) for the phase with this parity; warp-uniform result.
__device__ __forceinline__ bool tile_wait(uint32_t bar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < kTileWaitPolls; ++it) {
        if (!done)
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(bar), "r"(parity), "r"(kTileWaitHintNs)
                : "memory");
        if (__all_sync(FULL, done != 0)) return true;
    }
    return false;
}

// Tile copies of one block: descriptors (kernel parameters), the warp's
// mbarrier and the shared word with the parity of its next phase.
struct TileReq {
    const TileMaps* maps;   // nullptr: plain loads
    unsigned* status;
    unsigned bytes;         // bytes expected per block
    uint32_t bar;
    uint32_t* parity;
};

// a1 (plain loads, or from the tile in shared memory): raw values of column
// `lane` of the support, 0 where unknown; returns the known bits (bit m:
// pixel (m, lane)).  Pixels outside the image are unknown.
template <typename T>
__device__ __forceinline__ unsigned load_support(const ImageArgs& a, int y0, int x0, int lane,
                                                 const unsigned char* tile, T (&zr)[S]) {
    unsigned known = 0;
    if (tile != nullptr) {
        const float* ti = reinterpret_cast<const float*>(tile) + (x0 & 3) + lane;
        const unsigned char* tm = tile + kTileImgBytes + (x0 & 15) + lane;
#pragma unroll
        for (int m = 0; m < S; ++m) {
            const bool kn = tm[m * kTileMaskCols] != 0;
            const float fv = ti[m * kTileImgCols];
            zr[m] = kn ? T(fv) : T(0);   // select: unknown values never enter arithmetic
            known |= kn ? (1u << m) : 0u;
        }
        __syncwarp();   // the tile is consumed before the W area is reused
        return known;
    }
    const int xc = x0 + lane;
    const bool xin = (unsigned)xc < (unsigned)a.W;
#pragma unroll
    for (int m = 0; m < S; ++m) {
        const int y = y0 + m;
        bool kn = false;
        float fv = 0.f;
        if (xin && (unsigned)y < (unsigned)a.H) {
            const size_t off = (size_t)y * a.pitch + xc;
            kn = __ldg(a.mask + off) != 0;
            fv = __ldg(a.img + off);
        }
        zr[m] = kn ? T(fv) : T(0);
        known |= kn ? (1u << m) : 0u;
    }
    return known;
}

// Re-use of reconstructed pixels (the sequential form of the original FSR,
// which Sec. II leaves out): blocks run in raster order, and an unknown pixel
// of an earlier block's target takes part in later supports with its
// reconstruction and the weight delta rho^dist.  prev: the output image
// (same pitch), whose earlier targets are complete when the block runs.
struct ReuseCtx {
    const float* prev;
    float delta;
    int by, bx, B;
};

// a1 for the re-use form (plain loads): raw values of column `lane` of the
// support, 0 where neither known nor re-used; known bits in the return
// value, re-used bits (unknown pixels of blocks before (by, bx) in raster
// order) in `reused`.
template <typename T>
__device__ __forceinline__ unsigned load_support_reuse(const ImageArgs& a, const ReuseCtx& ru, int y0, int x0,
                                                       int lane, T (&zr)[S], unsigned& reused) {
    unsigned known = 0, reu = 0;
    const int xc = x0 + lane;
    const bool xin = (unsigned)xc < (unsigned)a.W;
    const int pbx = xin ? xc / ru.B : 0;
#pragma unroll
    for (int m = 0; m < S; ++m) {
        const int y = y0 + m;
        bool kn = false, re = false;
        float fv = 0.f;
        if (xin && (unsigned)y < (unsigned)a.H) {
            const size_t off = (size_t)y * a.pitch + xc;
            kn = __ldg(a.mask + off) != 0;
            const int pby = y / ru.B;
            re = !kn && (pby < ru.by || (pby == ru.by && pbx < ru.bx));
            // earlier targets were written by earlier launches: read through L2
            fv = kn ? __ldg(a.img + off) : (re ? __ldcg(ru.prev + off) : 0.f);
        }
        zr[m] = (kn || re) ? T(fv) : T(0);
        known |= kn ? (1u << m) : 0u;
        reu |= re ? (1u << m) : 0u;
    }
    reused = reu;
    return known;
}

// a1-a3 up to the packed spectrum: load the support (lane n = column n),
// weight it and transform z = x + j alpha w.  On return (when some pixel is
// known) lane k holds Z[k][0..31] = F2{z} row k in zr/zi; inv2alpha =
// 1 / (2 alpha); swd: sum of w in FP64 (precision study only).  Wd: this
// warp's scratch (the support tile and the transpose pass through it).
template <typename T, Dft DFT, bool REUSE = false, class TC = NoTc>
__device__ __forceinline__ bool transform_block(const ImageArgs& a, int y0, int x0, int lane,
                                                const T* __restrict__ sw0,
                                                typename Vec2<T>::type* Wd, TC* tc,
                                                const unsigned char* tile,
                                                T (&zr)[S], T (&zi)[S], BlockState<T>& st, T& inv2alpha_out,
                                                double& swd_out, const ReuseCtx* ru = nullptr) {
    using T2 = typename Vec2<T>::type;
    unsigned reused = 0;
    unsigned known;
    if constexpr (REUSE) known = load_support_reuse<T>(a, *ru, y0, x0, lane, zr, reused);
    else known = load_support<T>(a, y0, x0, lane, tile, zr);
    // Eq. (5): w0 on known pixels, delta w0 on re-used ones, 0 elsewhere
    auto weight = [&](int m) -> T {
        if constexpr (REUSE)
            return ((known >> m) & 1u) ? sw0[m * S + lane]
                                       : (((reused >> m) & 1u) ? T(ru->delta) * sw0[m * S + lane] : T(0));
        else
            return ((known >> m) & 1u) ? sw0[m * S + lane] : T(0);
    };
    const unsigned avail = known | reused;
    T sw = T(0), sfw = T(0);
    double swd = 0.0;   // precision study: W[0][0] = sum of w in FP64
#pragma unroll
    for (int m = 0; m < S; ++m) {
        const T w = weight(m);
        sw += w;
        sfw += w * zr[m];
        if constexpr (DFT != Dft::SIMT) swd += double(w);
    }
    if (__ballot_sync(FULL, avail != 0) == 0) return false;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(FULL, sw, o);
        sfw += __shfl_xor_sync(FULL, sfw, o);
        if constexpr (DFT != Dft::SIMT) swd += __shfl_xor_sync(FULL, swd, o);
    }
    const T mu = sfw / sw;   // any value works; the weighted mean makes Q[0][0] ~ 0
    st.mu = mu;

    // x = (f - mu) w on known pixels; alpha = 2^e >= max|f - mu| so that both
    // halves of z = x + j alpha w have one magnitude (W keeps FP32 precision
    // through the shared FFT); powers of two are undone exactly.
    unsigned dmax = 0;
#pragma unroll
    for (int m = 0; m < S; ++m) {
        const bool kn = (avail >> m) & 1u;
        const T w = weight(m);
        const T d = zr[m] - mu;
        zr[m] = kn ? d * w : T(0);
        zi[m] = w;
        const unsigned ab = __float_as_uint((float)d) & 0x7fffffffu;
        dmax = (kn && ab > dmax) ? ab : dmax;
    }
    dmax = __reduce_max_sync(FULL, dmax);
    unsigned aexp = (dmax >> 23) + 1u;             // exponent field of 2^e
    aexp = (dmax >= 0x00800000u && dmax < 0x7e000000u) ? aexp : 127u;
    const T alpha = T(__uint_as_float(aexp << 23));
    const T inv2alpha = T(__uint_as_float((253u - aexp) << 23));   // 1 / (2 alpha)
#pragma unroll
    for (int m = 0; m < S; ++m) zi[m] = zi[m] * alpha;

    if constexpr (DFT != Dft::SIMT) {
        // a3 on tensor cores (precision study); lane k ends with Z[k][0..31]
        tc->dft2(zr, zi, lane);
    } else {
        // a3: FFT over m (lane n holds column n)
        fft32<T>(zr, zi);
        // transpose through this warp's (not yet used) W area
        T2* tb = Wd;
        __syncwarp();
#pragma unroll
        for (int k = 0; k < S; ++k) {
            T2 v; v.x = zr[k]; v.y = zi[k];
            tb[k * TSTRIDE + lane] = v;
        }
        __syncwarp();
#pragma unroll
        for (int n = 0; n < S; ++n) {
            const T2 v = tb[lane * TSTRIDE + n];
            zr[n] = v.x; zi[n] = v.y;
        }
        __syncwarp();
        // FFT over n: lane k holds Z[k][0..31]
        fft32<T>(zr, zi);
    }
    inv2alpha_out = inv2alpha;
    swd_out = swd;
    return true;
}

// a1-a3: load the support (lane n = column n), weight it, transform it.
// On return (when some pixel is known) lane k holds Q[k][0..31] = F2{(f~-mu)w}
// row k in zr/zi and the W rows are in Wd (layout of WRow<T>).
template <typename T, int WS, Dft DFT, bool REUSE = false, class TC = NoTc>
__device__ __forceinline__ bool prepare_block(const ImageArgs& a, int y0, int x0, int lane,
                                              const T* __restrict__ sw0,
                                              typename Vec2<T>::type* Wd, TC* tc,
                                              const unsigned char* tile,
                                              T (&zr)[S], T (&zi)[S], BlockState<T>& st,
                                              const ReuseCtx* ru = nullptr) {
    using T2 = typename Vec2<T>::type;
    T inv2alpha;
    double swd;
    if (!transform_block<T, DFT, REUSE, TC>(a, y0, x0, lane, sw0, Wd, tc, tile, zr, zi, st, inv2alpha, swd, ru))
        return false;

    // Q[k][l] = (Z[k][l] + conj Z[-k][-l]) / 2,  W[k][l] = (Z[k][l] - conj Z[-k][-l]) / (2j alpha)
    const int src = (S - lane) & (S - 1);
    T2* wrow_out = Wd + lane * WS;
    T W0 = T(0);
#pragma unroll
    for (int l = 0; l <= S / 2; ++l) {
        const int l2 = (S - l) & (S - 1);
        const T cr = __shfl_sync(FULL, zr[l2], src);
        const T ci = __shfl_sync(FULL, zi[l2], src);
        T dr = cr, di = ci;
        if (l2 != l) {
            dr = __shfl_sync(FULL, zr[l], src);
            di = __shfl_sync(FULL, zi[l], src);
        }
        const T ar = zr[l], ai = zi[l];
        T2 w1;
        w1.x = (ai + ci) * inv2alpha;
        w1.y = (cr - ar) * inv2alpha;
        zr[l] = (ar + cr) * T(0.5);
        zi[l] = (ai - ci) * T(0.5);
        wrow_out[l] = w1;
        if (l + S < WS - 1) wrow_out[l + S] = w1;
        if (l == 0) W0 = w1.x;
        if (l2 != l) {
            const T br = zr[l2], bi = zi[l2];
            T2 w2;
            w2.x = (bi + di) * inv2alpha;
            w2.y = (dr - br) * inv2alpha;
            zr[l2] = (br + dr) * T(0.5);
            zi[l2] = (bi - di) * T(0.5);
            wrow_out[l2] = w2;
            if (l2 + S < WS - 1) wrow_out[l2 + S] = w2;
        }
    }
    st.W0 = __shfl_sync(FULL, W0, 0);
    // precision study: the normalisation of Eq. (10) uses W[0][0] summed in
    // FP64 from the weights, not the reduced-precision GEMM output
    if constexpr (DFT != Dft::SIMT) st.W0 = T(swd);
    __syncwarp();
    return true;
}

// R = a W + Q for one component (the DC-split representation); the same
// rounded operations everywhere, so every copy of a value is bit-identical.
template <typename T>
__device__ __forceinline__ void split_value(T ar, T ai, T wr, T wi, T qr, T qi, T& rr, T& ri) {
    rr = fma_rn(ar, wr, fma_rn(-ai, wi, qr));
    ri = fma_rn(ar, wi, fma_rn(ai, wr, qi));
}

// Eq. (12) for one component: R -= c W.
template <typename T>
__device__ __forceinline__ void residual_update(T& re, T& im, T wr, T wi, T cr, T ci) {
    re = fma_rn(-cr, wr, fma_rn(ci, wi, re));
    im = fma_rn(-cr, wi, fma_rn(-ci, wr, im));
}

// ---------------------------------------------------------------- FP32 loop
// Lane k holds Q[k][l] in zr[l], zi[l] and w_f[k][l] in wfr[min(l, 32-l)].
// Every pass leaves in g[j] the maximum of the objective over the group of
// GS components GS*j .. GS*j+GS-1 of the lane's row (short, independent max
// chains); the argmax then needs only the one group that holds the block
// maximum.

constexpr int WS32 = WRow<float>::stride;
constexpr int NG = 2;            // groups per row
constexpr int GS = S / NG;       // components per group
static_assert(GS % 4 == 0 && GS <= 16, "a group is published as GS / 4 float4 stores");

__device__ __forceinline__ float wf_at(const float (&wfr)[S / 2 + 1], int l) {
    return wfr[l <= S / 2 ? l : S - l];
}

__device__ __forceinline__ void group_max(float (&g)[NG], int i, float o0, float o1) {
    // pair i = components 2i, 2i+1 belongs to group i / (GS / 2)
    constexpr int PPG = GS / 2;
    if (i % PPG == 0) g[i / PPG] = fmaxf(o0, o1);
    else g[i / PPG] = max3(g[i / PPG], o0, o1);
}

// maximum over the groups
__device__ __forceinline__ float groups_max(const float (&g)[NG]) {
    if constexpr (NG == 8) return max3(max3(g[0], g[1], g[2]), max3(g[3], g[4], g[5]), fmaxf(g[6], g[7]));
    else if constexpr (NG == 4) return fmaxf(max3(g[0], g[1], g[2]), g[3]);
    else return fmaxf(g[0], g[1]);
}

// objective pass of R = a W + Q over the unshifted row k (DC phase)
__device__ __forceinline__ void pass_split_objective(const float (&zr)[S], const float (&zi)[S],
                                                     const float (&wfr)[S / 2 + 1], const float2* wrow,
                                                     float ar, float ai, float (&g)[NG]) {
    const float4* p = reinterpret_cast<const float4*>(wrow);
#pragma unroll
    for (int i = 0; i < S / 2; ++i) {
        const float4 w = p[i];
        float r0r, r0i, r1r, r1i;
        split_value(ar, ai, w.x, w.y, zr[2 * i], zi[2 * i], r0r, r0i);
        split_value(ar, ai, w.z, w.w, zr[2 * i + 1], zi[2 * i + 1], r1r, r1i);
        group_max(g, i, objective<float>(r0r, r0i, wf_at(wfr, 2 * i)),
                  objective<float>(r1r, r1i, wf_at(wfr, 2 * i + 1)));
    }
}

// fold a W into Q (end of the DC phase)
__device__ __forceinline__ void pass_fold(float (&zr)[S], float (&zi)[S], const float2* wrow,
                                          float ar, float ai) {
    const float4* p = reinterpret_cast<const float4*>(wrow);
#pragma unroll
    for (int i = 0; i < S / 2; ++i) {
        const float4 w = p[i];
        split_value(ar, ai, w.x, w.y, zr[2 * i], zi[2 * i], zr[2 * i], zi[2 * i]);
        split_value(ar, ai, w.z, w.w, zr[2 * i + 1], zi[2 * i + 1], zr[2 * i + 1], zi[2 * i + 1]);
    }
}

// Eq. (12) with the shifted row W[(k-u)][(l-v) mod 32], then the objective.
// Components 16h .. 16h+15 (h = 0, 1) read the 16 consecutive stored entries
// starting at (32 - v + 16h) mod 32 of row k-u, which never wrap in the
// 48-entry row.  For odd offsets the 16-byte loads start one entry earlier
// and each component takes the upper half of one load and the lower half of
// the next.
template <bool ODD>
__device__ __forceinline__ void half_update(float (&zr)[S], float (&zi)[S], const float (&wfr)[S / 2 + 1],
                                            const float2* base, int h, float cr, float ci, float (&g)[NG]) {
    const float4* p = reinterpret_cast<const float4*>(ODD ? base - 1 : base);
    float4 prev = ODD ? p[0] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < S / 4; ++j) {
        const int i = 8 * h + j;     // pair index: components 2i, 2i+1
        float w0r, w0i, w1r, w1i;
        if (ODD) {
            const float4 next = p[j + 1];
            w0r = prev.z; w0i = prev.w; w1r = next.x; w1i = next.y;
            prev = next;
        } else {
            const float4 w = p[j];
            w0r = w.x; w0i = w.y; w1r = w.z; w1i = w.w;
        }
        residual_update(zr[2 * i], zi[2 * i], w0r, w0i, cr, ci);
        residual_update(zr[2 * i + 1], zi[2 * i + 1], w1r, w1i, cr, ci);
        group_max(g, i, objective<float>(zr[2 * i], zi[2 * i], wf_at(wfr, 2 * i)),
                  objective<float>(zr[2 * i + 1], zi[2 * i + 1], wf_at(wfr, 2 * i + 1)));
    }
}

template <bool ODD>
__device__ __forceinline__ void pass_update(float (&zr)[S], float (&zi)[S], const float (&wfr)[S / 2 + 1],
                                            const float2* row, int s, float cr, float ci, float (&g)[NG]) {
    half_update<ODD>(zr, zi, wfr, row + s, 0, cr, ci, g);
    half_update<ODD>(zr, zi, wfr, row + ((s + S / 2) & (S - 1)), 1, cr, ci, g);
}

// Conjugate-pair ablation (the original FSR's real model): R -= c W1 + c* W2
// with W1 = W[k-u][l-v], W2 = W[k+u][l+v], formed from the sum and the
// difference of the two entries so that the update of (-k,-l) is the exact
// conjugate of that of (k,l) (R stays exactly Hermitian).
__device__ __forceinline__ void pair_update(float& re, float& im, float w1r, float w1i, float w2r, float w2i,
                                            float cr, float ci) {
    const float sr = w1r + w2r, si = w1i + w2i;
    const float dr = w1r - w2r, di = w1i - w2i;
    re = fma_rn(-cr, sr, fma_rn(ci, di, re));
    im = fma_rn(-cr, si, fma_rn(-ci, dr, im));
}

template <bool ODD>
__device__ __forceinline__ void half_update_pair(float (&zr)[S], float (&zi)[S], const float (&wfr)[S / 2 + 1],
                                                 const float2* base1, const float2* base2, int h, float cr,
                                                 float ci, float (&g)[NG]) {
    const float4* p1 = reinterpret_cast<const float4*>(ODD ? base1 - 1 : base1);
    const float4* p2 = reinterpret_cast<const float4*>(ODD ? base2 - 1 : base2);
    float4 prev1 = ODD ? p1[0] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 prev2 = ODD ? p2[0] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < S / 4; ++j) {
        const int i = 8 * h + j;
        float4 a, b;   // (entry 2i, entry 2i+1) of each row
        if (ODD) {
            const float4 n1 = p1[j + 1], n2 = p2[j + 1];
            a = make_float4(prev1.z, prev1.w, n1.x, n1.y);
            b = make_float4(prev2.z, prev2.w, n2.x, n2.y);
            prev1 = n1;
            prev2 = n2;
        } else {
            a = p1[j];
            b = p2[j];
        }
        pair_update(zr[2 * i], zi[2 * i], a.x, a.y, b.x, b.y, cr, ci);
        pair_update(zr[2 * i + 1], zi[2 * i + 1], a.z, a.w, b.z, b.w, cr, ci);
        group_max(g, i, objective<float>(zr[2 * i], zi[2 * i], wf_at(wfr, 2 * i)),
                  objective<float>(zr[2 * i + 1], zi[2 * i + 1], wf_at(wfr, 2 * i + 1)));
    }
}

// Row k reads row1 = W[k-u] from column s1 = -v and row2 = W[k+u] from
// column s2 = v (mod 32); s1 and s2 have the parity of v.
template <bool ODD>
__device__ __forceinline__ void pass_update_pair(float (&zr)[S], float (&zi)[S], const float (&wfr)[S / 2 + 1],
                                                 const float2* row1, int s1, const float2* row2, int s2,
                                                 float cr, float ci, float (&g)[NG]) {
    half_update_pair<ODD>(zr, zi, wfr, row1 + s1, row2 + s2, 0, cr, ci, g);
    half_update_pair<ODD>(zr, zi, wfr, row1 + ((s1 + S / 2) & (S - 1)), row2 + ((s2 + S / 2) & (S - 1)), 1, cr,
                          ci, g);
}

// (u, v) is its own conjugate: 2u = 2v = 0 mod S
__device__ __forceinline__ bool self_conjugate(int u, int v) { return ((u | v) & (S / 2 - 1)) == 0; }

// Lane u writes components GS*j .. GS*j+GS-1 of its row to rowbuf[0..GS-1]
// (j uniform).
template <int J>
__device__ __forceinline__ void store_group(const float (&zr)[S], const float (&zi)[S], float4* pub) {
    if constexpr (J < NG) {
#pragma unroll
        for (int t = 0; t < GS / 2; ++t) {
            const int c = GS * J + 2 * t;
            pub[t] = make_float4(zr[c], zi[c], zr[c + 1], zi[c + 1]);
        }
    }
}

__device__ __forceinline__ void publish_group(const float (&zr)[S], const float (&zi)[S], int j,
                                              bool mine, float2* rowbuf) {
    float4* pub = reinterpret_cast<float4*>(rowbuf);
    switch (j) {
#define FSR_PUB_CASE(J)                               \
        case J:                                       \
            if (mine) store_group<J>(zr, zi, pub);    \
            break;
        FSR_PUB_CASE(0) FSR_PUB_CASE(1) FSR_PUB_CASE(2) FSR_PUB_CASE(3)
        FSR_PUB_CASE(4) FSR_PUB_CASE(5) FSR_PUB_CASE(6) FSR_PUB_CASE(7)
#undef FSR_PUB_CASE
        default: break;
    }
}

// a5: argmax with the lowest linear index on ties.  Returns (u, v) and R[u][v];
// SPLIT: the spectrum is R = a W + Q (DC phase).
struct Pick {
    int u, v;
    float Rr, Ri;
};

template <bool SPLIT>
__device__ __forceinline__ Pick argmax_pick(const float (&zr)[S], const float (&zi)[S], const float (&g)[NG],
                                            const float2* Wd, float2* rowbuf, const float* __restrict__ swf,
                                            float ar, float ai, int lane) {
    const float m = groups_max(g);
    const unsigned Mb = __reduce_max_sync(FULL, __float_as_uint(m));
    const unsigned bu = __ballot_sync(FULL, __float_as_uint(m) == Mb);
    const int u = __ffs(bu) - 1;
    // first group of lane u's row that holds the maximum
    int jg;
    if constexpr (NG == 2) {
        // a second ballot, independent of u: bit u says whether group 0 holds it
        const unsigned b0 = __ballot_sync(FULL, __float_as_uint(g[0]) == Mb);
        jg = ((b0 >> u) & 1u) ? 0 : 1;
    } else {
        jg = NG - 1;
#pragma unroll
        for (int j = NG - 2; j >= 0; --j) jg = (__float_as_uint(g[j]) == Mb) ? j : jg;
        jg = __shfl_sync(FULL, jg, u);
    }
    publish_group(zr, zi, jg, lane == u, rowbuf);
    __syncwarp();
    const int cl = GS * jg + (lane & (GS - 1));   // column examined by this lane
    const float2 q = rowbuf[lane & (GS - 1)];
    float rr = q.x, ri = q.y;
    if constexpr (SPLIT) {
        const float2 w = Wd[u * WS32 + cl];
        split_value(ar, ai, w.x, w.y, q.x, q.y, rr, ri);
    }
    const float o = objective<float>(rr, ri, swf[u * WFS + cl]);
    const int vl = __ffs(__ballot_sync(FULL, __float_as_uint(o) == Mb)) - 1;   // lanes 0..GS-1 lead
    Pick pk;
    pk.u = u;
    pk.v = GS * jg + vl;
    pk.Rr = __shfl_sync(FULL, rr, vl);
    pk.Ri = __shfl_sync(FULL, ri, vl);
    __syncwarp();
    return pk;
}

// The picks of one block in iteration order (precision study): the
// coefficient c = gamma p and the index u*S+v of every iteration.
struct PickList {
    float2* c;
    int16_t* idx;
};

// a6 for the pick of iteration nu: c = gamma p, p = R[u,v] / W[0,0]
// (Eqs. 10-11), formed as R[u,v] (gamma / W[0,0]) with the block constant
// cg = gamma / W[0,0] (the same rounding as gamma (R / W[0,0]) when gamma is
// a power of two); records the index and adds Re(c e^{+j2pi(um+vn)/S}) to the
// target pixels (sparse inverse of G).  DENSE (precision study): the pick is
// appended to the block's pick list instead; after the loop the list gives
// the dense coefficient array (G of Eq. 11 divided by S^2), whose inverse
// transform runs on tensor cores.
template <int B, bool DENSE>
__device__ __forceinline__ void record_pick(const Pick& pk, float cg, int nu, int lane,
                                            int16_t* seq, const float2* __restrict__ scs,
                                            const int (&pm)[TargetPix<B>::P], const int (&pn)[TargetPix<B>::P],
                                            float (&gacc)[TargetPix<B>::P], const PickList* pl, float& cr,
                                            float& ci, bool pair = false) {
    cr = pk.Rr * cg;
    ci = pk.Ri * cg;
    if (seq != nullptr && lane == 0) seq[nu] = (int16_t)(pk.u * S + pk.v);
    if constexpr (DENSE) {
        if (lane == 0) {
            pl->c[nu] = make_float2(cr, ci);
            pl->idx[nu] = (int16_t)(pk.u * S + pk.v);
        }
    } else {
        // a conjugate pair adds Re(c e^{+j theta}) + Re(c* e^{-j theta}) = 2 Re(c e^{+j theta})
        const float gr = pair ? 2.f * cr : cr, gi = pair ? 2.f * ci : ci;
#pragma unroll
        for (int q2 = 0; q2 < TargetPix<B>::P; ++q2) {
            const float2 cs = scs[(pk.u * pm[q2] + pk.v * pn[q2]) & (S - 1)];
            gacc[q2] = fma_rn(gr, cs.x, fma_rn(-gi, cs.y, gacc[q2]));
        }
    }
}

// a4-a8 for one block.  Two loops: while only the DC basis image is
// selected, R stays a W + Q (DC phase); at the first other selection a W is
// folded into Q and the plain loop runs the remaining iterations.  The
// residual update after the last selection is not needed and not done.
template <int B, bool DENSE = false, bool CONJ = false>
__device__ __forceinline__ void iterate(float (&zr)[S], float (&zi)[S], float2* Wd, float2* rowbuf,
                                        const float* __restrict__ swf, const float2* __restrict__ scs,
                                        const BlockState<float>& st, float gamma, int K, int L, int lane,
                                        int16_t* seq, float (&gacc)[TargetPix<B>::P], const PickList* gd = nullptr) {
    constexpr int P = TargetPix<B>::P;
    if (K <= 0) return;
    float wfr[S / 2 + 1];
#pragma unroll
    for (int l = 0; l <= S / 2; ++l) wfr[l] = swf[lane * WFS + l];
    int pm[P], pn[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        pm[q] = L + (lane + 32 * q) / B;
        pn[q] = L + (lane + 32 * q) % B;
    }
    const float cg = gamma * (1.f / st.W0);
    const float2* wrow_k = Wd + lane * WS32;
    float g[NG];
    float cr, ci;
    Pick pk;
    int nu = 0;

    // ---- DC phase: R = a W + Q ----
    {
        float ar = st.mu, ai = 0.f;
        pass_split_objective(zr, zi, wfr, wrow_k, ar, ai, g);
        for (;;) {
            pk = argmax_pick<true>(zr, zi, g, Wd, rowbuf, swf, ar, ai, lane);
            record_pick<B, DENSE>(pk, cg, nu, lane, seq, scs, pm, pn, gacc, gd, cr, ci,
                                  CONJ && !self_conjugate(pk.u, pk.v));
            if (++nu == K) return;
            if ((pk.u | pk.v) != 0) break;
            ar -= cr;
            ai -= ci;
            pass_split_objective(zr, zi, wfr, wrow_k, ar, ai, g);
        }
        pass_fold(zr, zi, wrow_k, ar, ai);
    }

    // ---- a7 (Eq. 12) for the last pick, then a4-a6 of the next iteration ----
    for (;;) {
        const int s = (S - pk.v) & (S - 1);
        const float2* row = Wd + ((lane - pk.u) & (S - 1)) * WS32;
        if (CONJ && !self_conjugate(pk.u, pk.v)) {
            const float2* row2 = Wd + ((lane + pk.u) & (S - 1)) * WS32;
            if (s & 1) pass_update_pair<true>(zr, zi, wfr, row, s, row2, pk.v, cr, ci, g);
            else pass_update_pair<false>(zr, zi, wfr, row, s, row2, pk.v, cr, ci, g);
        } else {
            if (s & 1) pass_update<true>(zr, zi, wfr, row, s, cr, ci, g);
            else pass_update<false>(zr, zi, wfr, row, s, cr, ci, g);
        }
        pk = argmax_pick<false>(zr, zi, g, Wd, rowbuf, swf, 0.f, 0.f, lane);
        record_pick<B, DENSE>(pk, cg, nu, lane, seq, scs, pm, pn, gacc, gd, cr, ci,
                              CONJ && !self_conjugate(pk.u, pk.v));
        if (++nu == K) return;
    }
}

// ---------------------------------------------------------------- FP64 loop
// The debug arithmetic: plain scalar loop with the same representation and
// selection rule, IEEE division for p.
template <int B, bool DENSE_UNUSED = false, bool CONJ = false>
__device__ __forceinline__ void iterate(double (&zr)[S], double (&zi)[S], double2* Wd, double2* rowbuf,
                                        const double* __restrict__ swf, const double2* __restrict__ scs,
                                        const BlockState<double>& st, double gamma, int K, int L, int lane,
                                        int16_t* seq, double (&gacc)[TargetPix<B>::P]) {
    constexpr int P = TargetPix<B>::P;
    constexpr int WS = WRow<double>::stride;
    double wfr[S / 2 + 1];
#pragma unroll
    for (int l = 0; l <= S / 2; ++l) wfr[l] = swf[lane * WFS + l];
    int pm[P], pn[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        pm[q] = L + (lane + 32 * q) / B;
        pn[q] = L + (lane + 32 * q) % B;
    }
    const double2* wrow_k = Wd + lane * WS;
    double ar = st.mu, ai = 0.0;
    bool split = true;
    double m = 0.0;
#pragma unroll
    for (int l = 0; l < S; ++l) {
        double rr, ri;
        split_value(ar, ai, wrow_k[l].x, wrow_k[l].y, zr[l], zi[l], rr, ri);
        m = fmax(m, objective<double>(rr, ri, wfr[l <= S / 2 ? l : S - l]));
    }
    for (int nu = 0; nu < K; ++nu) {
        const double M = warp_max(m);
        const int u = __ffs(__ballot_sync(FULL, m == M)) - 1;
        if (lane == u) {
#pragma unroll
            for (int l = 0; l < S; ++l) { double2 t; t.x = zr[l]; t.y = zi[l]; rowbuf[l] = t; }
        }
        __syncwarp();
        const double2 q = rowbuf[lane];
        double rr = q.x, ri = q.y;
        if (split) split_value(ar, ai, Wd[u * WS + lane].x, Wd[u * WS + lane].y, q.x, q.y, rr, ri);
        const double o = objective<double>(rr, ri, swf[u * WFS + lane]);
        const int v = __ffs(__ballot_sync(FULL, o == M)) - 1;
        const double Rr = __shfl_sync(FULL, rr, v);
        const double Ri = __shfl_sync(FULL, ri, v);
        __syncwarp();
        const double cr = gamma * (Rr / st.W0);
        const double ci = gamma * (Ri / st.W0);
        if (seq != nullptr && lane == 0) seq[nu] = (int16_t)(u * S + v);
        const bool pair = CONJ && !self_conjugate(u, v);
        const double gr = pair ? 2.0 * cr : cr, gi = pair ? 2.0 * ci : ci;
#pragma unroll
        for (int q2 = 0; q2 < P; ++q2) {
            const double2 cs = scs[(u * pm[q2] + v * pn[q2]) & (S - 1)];
            gacc[q2] = fma_rn(gr, cs.x, fma_rn(-gi, cs.y, gacc[q2]));
        }
        if (split) {
            if ((u | v) == 0) {
                ar -= cr;
                ai -= ci;
                m = 0.0;
#pragma unroll
                for (int l = 0; l < S; ++l) {
                    double r1, r2;
                    split_value(ar, ai, wrow_k[l].x, wrow_k[l].y, zr[l], zi[l], r1, r2);
                    m = fmax(m, objective<double>(r1, r2, wfr[l <= S / 2 ? l : S - l]));
                }
                continue;
            }
#pragma unroll
            for (int l = 0; l < S; ++l)
                split_value(ar, ai, wrow_k[l].x, wrow_k[l].y, zr[l], zi[l], zr[l], zi[l]);
            split = false;
        }
        const double2* wrow = Wd + ((lane - u) & (S - 1)) * WS + ((S - v) & (S - 1));
        m = 0.0;
        if (pair) {
            // conjugate-pair ablation: R -= c W[k-u][l-v] + c* W[k+u][l+v]
            const double2* wrow2 = Wd + ((lane + u) & (S - 1)) * WS + (v & (S - 1));
#pragma unroll
            for (int l = 0; l < S; ++l) {
                const double2 w1 = wrow[l], w2 = wrow2[l];
                const double sr = w1.x + w2.x, si = w1.y + w2.y;
                const double dr = w1.x - w2.x, di = w1.y - w2.y;
                zr[l] = fma_rn(-cr, sr, fma_rn(ci, di, zr[l]));
                zi[l] = fma_rn(-cr, si, fma_rn(-ci, dr, zi[l]));
                m = fmax(m, objective<double>(zr[l], zi[l], wfr[l <= S / 2 ? l : S - l]));
            }
            continue;
        }
#pragma unroll
        for (int l = 0; l < S; ++l) {
            const double2 w = wrow[l];
            residual_update(zr[l], zi[l], w.x, w.y, cr, ci);
            m = fmax(m, objective<double>(zr[l], zi[l], wfr[l <= S / 2 ? l : S - l]));
        }
    }
}

// Shared-memory tables of one CTA: Eqs. (5) and (9) and cos/sin(2 pi t / S).
template <typename T>
__device__ __forceinline__ void cta_tables(const MethodArgs& mth, T* sw0, T* swf,
                                           typename Vec2<T>::type* scs) {
    using T2 = typename Vec2<T>::type;
    const T half = T(S) / T(2);
    for (int i = threadIdx.x; i < S * S; i += blockDim.x) {
        const int m = i / S, n = i % S;
        const T dm = T(m) - T(S - 1) / T(2), dn = T(n) - T(S - 1) / T(2);
        sw0[i] = pow(T(mth.rho), sqrt(dm * dm + dn * dn));
        T wfv = T(1);
        if (mth.freq_weight) {
            const T kt = half - fabs(T(m) - half), lt = half - fabs(T(n) - half);
            const T r = sqrt(kt * kt / T(S * S) + lt * lt / T(S * S));
            const T b = T(1) - sqrt(T(2)) * r;
            wfv = b * b;
        }
        swf[m * WFS + n] = wfv;
    }
    for (int t = threadIdx.x; t < S; t += blockDim.x) {
        T2 v;
        v.x = T(cos_2pi32(t));
        v.y = T(sin_2pi32(t));
        scs[t] = v;
    }
}

// A support without a known pixel: no iterations (g = 0), the selection
// sequence is -1, and the block is counted (reading: W[0][0] = 0).
__device__ __forceinline__ void empty_block(int16_t* seq, int K, unsigned long long* empty) {
    if (seq != nullptr)
        for (int nu = 0; nu < K; ++nu) seq[nu] = -1;
    if (empty != nullptr) atomicAdd(empty, 1ull);
}

// Everything of one target block: a1-a3 (prepare), a4-a8 (iterate), a9.
// With a tile context the support comes in by TMA; returns false when the
// bounded wait for it gave up (the warp then stops taking blocks).
template <typename T, int B, bool CONJ = false, bool REUSE = false>
__device__ __forceinline__ bool process_block(const ImageArgs& im, long long blk, int L, T gamma,
                                              const T* sw0, const T* swf, const typename Vec2<T>::type* scs,
                                              typename Vec2<T>::type* Wd, typename Vec2<T>::type* rowbuf,
                                              const TileReq& tr, unsigned long long* empty, int lane,
                                              float delta = 0.f) {
    constexpr int P = TargetPix<B>::P;
    const int by = (int)(blk / im.nbx);
    const int bx = (int)(blk - (long long)by * im.nbx);
    const int y0 = by * B - L, x0 = bx * B - L;

    const unsigned char* tile = nullptr;
    if (tr.maps != nullptr) {
        __syncwarp();   // every lane is done with the W area of the previous block
        if (lane == 0) tile_issue(tr.maps, smem_addr(Wd), tr.bar, y0, x0, tr.bytes);
        const uint32_t parity = *tr.parity;
        if (!tile_wait(tr.bar, parity)) {
            if (lane == 0) atomicOr(tr.status, kStatusTileWait);
            return false;
        }
        __syncwarp();
        if (lane == 0) *tr.parity = parity ^ 1u;
        tile = reinterpret_cast<const unsigned char*>(Wd);
    }

    T zr[S], zi[S];
    BlockState<T> st;
    T gacc[P];
#pragma unroll
    for (int q = 0; q < P; ++q) gacc[q] = T(0);

    int16_t* seq = im.seq ? im.seq + (size_t)blk * im.K : nullptr;
    {
        ReuseCtx ru;
        if constexpr (REUSE) {
            ru.prev = im.out;
            ru.delta = delta;
            ru.by = by;
            ru.bx = bx;
            ru.B = B;
        }
        if (prepare_block<T, SmemLayout<T>::WS, Dft::SIMT, REUSE>(im, y0, x0, lane, sw0, Wd, (NoTc*)nullptr, tile,
                                                                   zr, zi, st, REUSE ? &ru : nullptr)) {
            iterate<B, false, CONJ>(zr, zi, Wd, rowbuf, swf, scs, st, gamma, im.K, L, lane, seq, gacc);
            __syncwarp();   // W area free for the next block
        } else if (lane == 0) {
            empty_block(seq, im.K, empty);
        }
    }

    // ---- a9: write-back of the B x B target ----
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int pidx = lane + 32 * q;
        if (pidx < B * B) {
            const int ty = by * B + pidx / B, tx = bx * B + pidx % B;
            if (ty < im.H && tx < im.W) {
                const size_t off = (size_t)ty * im.pitch + tx;
                const bool kn = __ldg(im.mask + off) != 0;
                im.out[off] = kn ? __ldg(im.img + off) : (float)gacc[q];
            }
        }
    }
    return true;
}

// Register budget: FP32 CTAs are sized so that 16 warps share an SM (at most
// 128 registers per thread), FP64 runs one CTA per SM.
template <typename T, int WARPS> struct MinBlocks { static constexpr int value = 1; };
template <int WARPS> struct MinBlocks<float, WARPS> { static constexpr int value = WARPS < 16 ? 16 / WARPS : 1; };

template <typename T, int B, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, MinBlocks<T, WARPS>::value)
fsr_blocks_kernel(const __grid_constant__ KernelArgs a) {
    using T2 = typename Vec2<T>::type;
    using Lay = SmemLayout<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    T* sw0 = reinterpret_cast<T*>(smem + Lay::w0_off);
    T* swf = reinterpret_cast<T*>(smem + Lay::wf_off);
    T2* scs = reinterpret_cast<T2*>(smem + Lay::cs_off);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    T2* Wd = reinterpret_cast<T2*>(smem + Lay::warp0_off + Lay::per_warp * warp);
    T2* rowbuf = Wd + Lay::w_elems;

    cta_tables<T>(a.mth, sw0, swf, scs);
    __syncthreads();

    // tile copies need 128-byte aligned destinations (kept by the layout)
    const bool tiles = a.tiles && (smem_addr(smem) & 127u) == 0;
    if (tiles) {
        if (lane == 0) {
            tile_bar_init(smem_addr(smem + Lay::bar_off(WARPS) + 8 * warp));
            reinterpret_cast<uint32_t*>(smem + Lay::parity_off(WARPS))[warp] = 0;
        }
        __syncwarp();
    }

    const T gamma = T(a.mth.gamma);
    for (;;) {
        unsigned long long next = 0;
        if (lane == 0) next = atomicAdd(a.work, 1ull);
        const long long blk = (long long)__shfl_sync(FULL, next, 0);
        if (blk >= a.nblocks) break;
        const int wq = threadIdx.x >> 5;
        TileReq tr;
        tr.maps = tiles ? &a.maps : nullptr;
        tr.status = a.status;
        tr.bytes = kTileBytes + (unsigned)a.tx_extra;
        tr.bar = smem_addr(smem + Lay::bar_off(WARPS) + 8 * wq);
        tr.parity = reinterpret_cast<uint32_t*>(smem + Lay::parity_off(WARPS)) + wq;
        if (!process_block<T, B>(a.im, blk, a.mth.L, gamma, sw0, swf, scs, Wd, rowbuf, tr, a.empty, lane))
            break;
    }
    // the last warp of the launch leaves the counter at zero for the next one
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(a.work + 1, 1ull) == (unsigned long long)gridDim.x * WARPS - 1) {
            atomicExch(a.work, 0ull);
            atomicExch(a.work + 1, 0ull);
        }
    }
}

// Batch form: every warp takes `chunk` consecutive entries of the block list
// at a time; images are ordered by decreasing K so the long blocks start first.
// ONE_ROUND: short-lived CTAs (a warp takes one chunk; the grid is sized to
// the work), used by the serving loop so that the CTAs of a launch on a
// higher-priority stream are scheduled as soon as running CTAs finish.
template <typename T, int B, int WARPS, bool CONJ = false, bool ONE_ROUND = false>
__global__ void __launch_bounds__(WARPS * 32, MinBlocks<T, WARPS>::value)
fsr_batch_kernel(const BatchArgs a) {
    using T2 = typename Vec2<T>::type;
    using Lay = SmemLayout<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    T* sw0 = reinterpret_cast<T*>(smem + Lay::w0_off);
    T* swf = reinterpret_cast<T*>(smem + Lay::wf_off);
    T2* scs = reinterpret_cast<T2*>(smem + Lay::cs_off);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    T2* Wd = reinterpret_cast<T2*>(smem + Lay::warp0_off + Lay::per_warp * warp);
    T2* rowbuf = Wd + Lay::w_elems;

    cta_tables<T>(a.mth, sw0, swf, scs);
    __syncthreads();

    // tile copies need 128-byte aligned destinations (kept by the layout)
    const bool tiles = a.maps != nullptr && (smem_addr(smem) & 127u) == 0;
    if (tiles) {
        if (lane == 0) {
            tile_bar_init(smem_addr(smem + Lay::bar_off(WARPS) + 8 * warp));
            reinterpret_cast<uint32_t*>(smem + Lay::parity_off(WARPS))[warp] = 0;
        }
        __syncwarp();
    }

    const T gamma = T(a.mth.gamma);
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.counter, (unsigned long long)a.chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= (unsigned long long)a.total) break;
        const long long end = min((long long)base + a.chunk, a.total);
        bool ok = true;
        for (long long item = (long long)base; item < end && ok; ++item) {
            // image of this entry: last i with first[i] <= item
            int lo = 0, hi = a.n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(a.first + mid) <= item) lo = mid;
                else hi = mid - 1;
            }
            const ImageArgs im = a.images[lo];
            TileReq tr;
            tr.maps = (tiles && im.tiles) ? a.maps + lo : nullptr;
            tr.status = a.status;
            tr.bytes = kTileBytes + (unsigned)a.tx_extra;
            tr.bar = smem_addr(smem + Lay::bar_off(WARPS) + 8 * warp);
            tr.parity = reinterpret_cast<uint32_t*>(smem + Lay::parity_off(WARPS)) + warp;
            ok = process_block<T, B, CONJ>(im, item - __ldg(a.first + lo), a.mth.L, gamma, sw0, swf, scs, Wd,
                                           rowbuf, tr, a.empty, lane);
        }
        if (!ok) break;   // a tile wait gave up: this warp takes no more blocks
        if constexpr (ONE_ROUND) break;
    }
}

// Re-use form: one launch per wavefront t of the raster order.  Block
// (by, bx) runs in wavefront t = a by + bx with a = ceil(L / B) + 1, so every
// block of the raster order before it whose target meets its support (rows
// by - ceil(L/B) .. by, columns up to bx + ceil(L/B)) ran in an earlier
// launch, and no two blocks of one launch touch each other's supports.
// One image's blocks on wavefront t: block rows by_lo .. by_lo + count - 1
// (bx = t - a by); they are the launch's blocks first .. first + count - 1.
struct ReuseSeg {
    ImageArgs im;
    int by_lo, count, first;
};
constexpr int kReuseSegs = 48;   // images per launch (the launch parameters stay below 4 KB)

// The parameters of one wavefront launch, with room for NSEG images: a
// single image launches with NSEG = 1 (about 100 bytes of parameters per
// launch instead of 3.5 KB).
template <int NSEG>
struct ReuseLaunchN {
    MethodArgs mth;
    float delta;            // re-use weight (0 < delta <= 1)
    int t;                  // wavefront
    int slope;              // a = ceil(L / B) + 1
    int nseg, total;        // segments, and the blocks they hold
    unsigned long long* empty;
    ReuseSeg seg[NSEG];
};
using ReuseLaunch = ReuseLaunchN<kReuseSegs>;
static_assert(sizeof(ReuseLaunch) <= 4096, "re-use launch parameters must fit the 4 KB parameter space");

// the first segment of a launch, as a one-image launch
inline ReuseLaunchN<1> one_image(const ReuseLaunch& a) {
    ReuseLaunchN<1> b;
    b.mth = a.mth;
    b.delta = a.delta;
    b.t = a.t;
    b.slope = a.slope;
    b.nseg = 1;
    b.total = a.seg[0].count;
    b.empty = a.empty;
    b.seg[0] = a.seg[0];
    return b;
}

template <typename T, int B, int WARPS, int NSEG>
__global__ void __launch_bounds__(WARPS * 32, MinBlocks<T, WARPS>::value)
fsr_reuse_kernel(const __grid_constant__ ReuseLaunchN<NSEG> a) {
    using T2 = typename Vec2<T>::type;
    using Lay = SmemLayout<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    T* sw0 = reinterpret_cast<T*>(smem + Lay::w0_off);
    T* swf = reinterpret_cast<T*>(smem + Lay::wf_off);
    T2* scs = reinterpret_cast<T2*>(smem + Lay::cs_off);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    T2* Wd = reinterpret_cast<T2*>(smem + Lay::warp0_off + Lay::per_warp * warp);
    T2* rowbuf = Wd + Lay::w_elems;
    cta_tables<T>(a.mth, sw0, swf, scs);
    __syncthreads();
    // Launched as a programmatic dependent of the previous wavefront: the
    // tables above overlap its end; nothing of the image or the output is
    // read before it has completed and its writes are visible.  The next
    // wavefront may then start its own tables.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int j = blockIdx.x * WARPS + warp;
    if (j >= a.total) return;
    TileReq tr;
    tr.maps = nullptr;
    if constexpr (NSEG == 1) {
        // one image: its fields at fixed offsets of the parameter space
        const int by = a.seg[0].by_lo + j;
        const int bx = a.t - a.slope * by;
        process_block<T, B, false, true>(a.seg[0].im, (long long)by * a.seg[0].im.nbx + bx, a.mth.L,
                                         T(a.mth.gamma), sw0, swf, scs, Wd, rowbuf, tr, a.empty, lane, a.delta);
    } else {
        int s = 0;   // the segment (image) of block j
        while (s + 1 < a.nseg && a.seg[s + 1].first <= j) ++s;
        const ReuseSeg& sg = a.seg[s];
        const int by = sg.by_lo + (j - sg.first);
        const int bx = a.t - a.slope * by;
        process_block<T, B, false, true>(sg.im, (long long)by * sg.im.nbx + bx, a.mth.L, T(a.mth.gamma), sw0, swf,
                                         scs, Wd, rowbuf, tr, a.empty, lane, a.delta);
    }
}

}  // namespace fsrk
