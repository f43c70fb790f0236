// FP64 FSR with the 4 x 4 support (S = 4: B = 4 with L = 0, or B = 2 with
// L = 1), the smallest support of the support-size study (Sec. IV, Fig. 3);
// FP32 at S = 4 runs the group kernel of fsr_group.cu.  One
// half-warp per block: lane t of the half holds pixel (t / 4, t % 4) and
// spectrum component (k, l) = (t / 4, t % 4).  The 2-D DFTs of Eq. (7) are
// direct sums over the 16 pixels, fetched by shuffles, with the exact fourth
// roots of unity (so R_w and W are exactly Hermitian and the ties of the
// first iteration are exact).  The argmax of Eq. (8) is a butterfly of
// (objective, index) pairs inside the half that keeps the lowest linear
// index on ties; p of Eq. (10) and the shifted W[k-u][l-v] of Eq. (12) are
// read from the lanes that hold them.  Re g (Eq. 11, sparse inverse) is
// accumulated at each lane's own pixel.  No shared memory.
#include "fsr_launch.h"

namespace fsrk {
namespace {

constexpr int kS4 = 4;
constexpr int kWarpsTiny = 8;

// cos(2 pi t / 4) and -sin(2 pi t / 4): e^{-j 2 pi t / 4} = 1, -j, -1, j
template <typename T>
__device__ __forceinline__ T cos4(int t) {
    t &= 3;
    return t == 0 ? T(1) : t == 2 ? T(-1) : T(0);
}
template <typename T>
__device__ __forceinline__ T msin4(int t) {
    t &= 3;
    return t == 1 ? T(-1) : t == 3 ? T(1) : T(0);
}

template <typename T, int B>
__device__ __forceinline__ void tiny_block(const ImageArgs& im, long long blk, bool valid, int Kmax, int L,
                                           const MethodArgs& mth, T gamma, unsigned long long* empty, int lane) {
    const int t = lane & 15, hb = lane & 16;   // lane in the half, first lane of the half
    const int m = t >> 2, n = t & 3;           // pixel (m, n); component (k, l) = (m, n)
    int by = 0, bx = 0;
    if (valid) {
        by = (int)(blk / im.nbx);
        bx = (int)(blk - (long long)by * im.nbx);
    }
    const int y = by * B - L + m, x = bx * B - L + n;
    bool kn = false;
    float fv = 0.f;
    size_t off = 0;
    if (valid && (unsigned)y < (unsigned)im.H && (unsigned)x < (unsigned)im.W) {
        off = (size_t)y * im.pitch + x;
        kn = __ldg(im.mask + off) != 0;
        fv = __ldg(im.img + off);
    }
    // a1, a2 (Eqs. 2, 5): weights on known pixels, weighted sampled signal
    const T dm = T(m) - T(kS4 - 1) / T(2), dn = T(n) - T(kS4 - 1) / T(2);
    const T w = kn ? T(pow(T(mth.rho), sqrt(dm * dm + dn * dn))) : T(0);
    const T xv = kn ? T(fv) * w : T(0);
    T wf = T(1);   // Eq. (9) at (k, l) = (m, n)
    if (mth.freq_weight) {
        const T half = T(kS4) / T(2);
        const T kt = half - fabs(T(m) - half), lt = half - fabs(T(n) - half);
        const T r = sqrt(kt * kt / T(kS4 * kS4) + lt * lt / T(kS4 * kS4));
        const T b = T(1) - sqrt(T(2)) * r;
        wf = b * b;
    }

    // a3: R[k][l] = sum x[m'][n'] e^{-j 2 pi (k m' + l n') / 4}, W likewise
    T Rr = T(0), Ri = T(0), Wr = T(0), Wi = T(0);
#pragma unroll
    for (int s = 0; s < kS4 * kS4; ++s) {
        const T xs = __shfl_sync(FULL, xv, hb + s);
        const T ws = __shfl_sync(FULL, w, hb + s);
        const int ph = m * (s >> 2) + n * (s & 3);
        const T c = cos4<T>(ph), sn = msin4<T>(ph);
        Rr = fma_rn(xs, c, Rr);
        Ri = fma_rn(xs, sn, Ri);
        Wr = fma_rn(ws, c, Wr);
        Wi = fma_rn(ws, sn, Wi);
    }
    const T W0 = __shfl_sync(FULL, Wr, hb);
    const unsigned known_bits = __ballot_sync(FULL, kn) & (0xFFFFu << hb);
    const bool active = valid && known_bits != 0u;
    const int Kh = valid ? im.K : 0;
    int16_t* seq = (valid && im.seq) ? im.seq + (size_t)blk * im.K : nullptr;
    if (valid && !active && t == 0) empty_block(seq, im.K, empty);
    const T invW0 = active ? T(1) / W0 : T(0);

    T gacc = T(0);   // Re g at this lane's pixel
    for (int nu = 0; nu < Kmax; ++nu) {   // uniform trip count over the warp
        const bool run = active && nu < Kh;
        // a4, a5: block maximum with the lowest linear index on ties
        T o = run ? objective<T>(Rr, Ri, wf) : T(-1);
        int idx = t;
#pragma unroll
        for (int s = 8; s > 0; s >>= 1) {
            const T oo = __shfl_xor_sync(FULL, o, s);
            const int oi = __shfl_xor_sync(FULL, idx, s);
            if (oo > o || (oo == o && oi < idx)) {
                o = oo;
                idx = oi;
            }
        }
        // a6 (Eqs. 10, 11)
        const T sr = __shfl_sync(FULL, Rr, hb + idx);
        const T si = __shfl_sync(FULL, Ri, hb + idx);
        const int u = idx >> 2, v = idx & 3;
        const T cr = gamma * (sr * invW0), ci = gamma * (si * invW0);
        // a7 (Eq. 12): R[k][l] -= c W[k-u][l-v]
        const int src = hb + (((m - u) & 3) << 2) + ((n - v) & 3);
        const T w1r = __shfl_sync(FULL, Wr, src);
        const T w1i = __shfl_sync(FULL, Wi, src);
        if (run) {
            if (seq != nullptr && t == 0) seq[nu] = (int16_t)(u * kS4 + v);
            const int ph = u * m + v * n;   // Re(c e^{+j 2 pi (u m + v n) / 4}) at this pixel
            gacc = fma_rn(cr, cos4<T>(ph), fma_rn(ci, msin4<T>(ph), gacc));
            residual_update(Rr, Ri, w1r, w1i, cr, ci);
        }
    }

    // a9: the target pixels of the support (m, n in [L, L + B))
    if (valid && m >= L && m < L + B && n >= L && n < L + B && (unsigned)y < (unsigned)im.H &&
        (unsigned)x < (unsigned)im.W)
        im.out[off] = kn ? fv : (float)gacc;
}

template <typename T, int B, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) fsr_tiny_kernel(const BatchArgs a) {
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4;
    const T gamma = T(a.mth.gamma);
    const long long take = 2ll * a.chunk;   // two blocks per warp and chunk step
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.counter, (unsigned long long)take);
        base = __shfl_sync(FULL, base, 0);
        if (base >= (unsigned long long)a.total) break;
        const long long end = min((long long)base + take, a.total);
        for (long long pair = (long long)base; pair < end; pair += 2) {
            const long long item = pair + half;
            const bool valid = item < end;
            ImageArgs im;
            im.img = nullptr;
            im.mask = nullptr;
            im.out = nullptr;
            im.seq = nullptr;
            im.H = im.W = im.pitch = im.nbx = im.K = im.tiles = 0;
            long long blk = 0;
            if (valid) {
                int lo = 0, hi = a.n - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (__ldg(a.first + mid) <= item) lo = mid;
                    else hi = mid - 1;
                }
                im = a.images[lo];
                blk = item - __ldg(a.first + lo);
            }
            const int Kh = valid ? im.K : 0;
            const int Kmax = max(Kh, __shfl_xor_sync(FULL, Kh, 16));
            tiny_block<T, B>(im, blk, valid, Kmax, a.mth.L, a.mth, gamma, a.empty, lane);
        }
    }
}

template <typename T, int B>
cudaError_t launch_one(const BatchArgs& a, int chunk, int sm_count, cudaStream_t stream) {
    int grid = 0;
    cudaError_t e = persistent_grid(fsr_tiny_kernel<T, B, kWarpsTiny>, kWarpsTiny, 0,
                                    (a.total + 2ll * chunk - 1) / (2ll * chunk), sm_count, &grid);
    if (e != cudaSuccess) return e;
    fsr_tiny_kernel<T, B, kWarpsTiny><<<grid, kWarpsTiny * 32, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tiny(const BatchArgs& a, int B, int chunk, int sm_count, cudaStream_t stream) {
    if (B == 4) return launch_one<double, 4>(a, chunk, sm_count, stream);
    if (B == 2) return launch_one<double, 2>(a, chunk, sm_count, stream);
    return cudaErrorNotSupported;
}

}  // namespace fsrk
