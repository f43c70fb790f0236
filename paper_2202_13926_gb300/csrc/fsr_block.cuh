// Per-block FSR on sm_103a: one warp owns one 32 x 32 support block.
//
// Sec. II / Sec. III of Regensky et al. (MMSP 2020), re-laid out for GB300:
//   * lane n first holds column n of the support, then (after one transpose
//     through shared memory) lane k holds row k of the spectrum: R_w[k][0..31]
//     lives in 64 registers of lane k for the whole iteration;
//   * the forward transform is one complex 32 x 32 DFT of z = x + j w
//     (x = f~ w, the weighted signal of Eq. 7, and w of Eq. 5), done as two
//     register-resident radix-2 FFT passes; R_w and W are separated with the
//     conjugate-symmetry identities, which makes both exactly Hermitian;
//   * W is kept in shared memory with every row stored twice in a row
//     (W[i][0..31] W[i][0..31]), so the circularly shifted row
//     W[(k-u) mod S][(l-v) mod S], l = 0..31 of Eqs. (12), (14), (15) is 32
//     consecutive entries starting at column (S - v) mod S: no index wrap;
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
#include <cuda_runtime.h>

namespace fsrk {

constexpr int S = 32;                 // support size of this kernel family
constexpr int WSTRIDE = 2 * S + 1;    // doubled W row + 1 pad (bank spread)
constexpr int TSTRIDE = S + 1;        // transpose buffer row stride
constexpr unsigned FULL = 0xffffffffu;

struct KernelArgs {
    const float* img;
    const uint8_t* mask;
    float* out;
    int16_t* seq;        // optional: N*K selected indices
    long long nblocks;   // N
    int H, W, pitch;     // image geometry (pitch in elements, shared by all three)
    int nbx;             // ceil(W / B)
    int L;               // border
    int K;               // iterations
    float rho, gamma;
    int freq_weight;
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

__device__ __forceinline__ float warp_max(float x) {
    // objective values are >= +0, so their bit patterns order like the values
    return __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(x)));
}
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(FULL, x, o));
    return x;
}

template <typename T>
struct SmemLayout {
    using T2 = typename Vec2<T>::type;
    // CTA-shared tables
    static constexpr size_t w0_off = 0;                                 // S*S T
    static constexpr size_t wf_off = w0_off + sizeof(T) * S * S;        // S*S T
    static constexpr size_t cs_off = wf_off + sizeof(T) * S * S;        // S T2
    static constexpr size_t warp0_off = cs_off + sizeof(T2) * S;
    // per warp: doubled W rows, then the published row
    static constexpr size_t w_elems = (size_t)S * WSTRIDE;
    static constexpr size_t per_warp = sizeof(T2) * (w_elems + S);
    static constexpr size_t bytes(int warps) { return warp0_off + per_warp * (size_t)warps; }
};

// Number of target pixels each lane accumulates for a B x B target.
template <int B> struct TargetPix { static constexpr int P = (B * B + 31) / 32; };

template <typename T, int B, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1)
fsr_blocks_kernel(const KernelArgs a) {
    using T2 = typename Vec2<T>::type;
    using Lay = SmemLayout<T>;
    constexpr int P = TargetPix<B>::P;
    extern __shared__ __align__(16) unsigned char smem[];
    T* sw0 = reinterpret_cast<T*>(smem + Lay::w0_off);
    T* swf = reinterpret_cast<T*>(smem + Lay::wf_off);
    T2* scs = reinterpret_cast<T2*>(smem + Lay::cs_off);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    T2* Wd = reinterpret_cast<T2*>(smem + Lay::warp0_off + Lay::per_warp * warp);
    T2* rowbuf = Wd + Lay::w_elems;

    // Tables of Eqs. (5) and (9) and cos/sin(2 pi t / S), per CTA.
    const T half = T(S) / T(2);
    for (int i = threadIdx.x; i < S * S; i += blockDim.x) {
        const int m = i / S, n = i % S;
        const T dm = T(m) - T(S - 1) / T(2), dn = T(n) - T(S - 1) / T(2);
        sw0[i] = pow(T(a.rho), sqrt(dm * dm + dn * dn));
        T wfv = T(1);
        if (a.freq_weight) {
            const T kt = half - fabs(T(m) - half), lt = half - fabs(T(n) - half);
            const T r = sqrt(kt * kt / T(S * S) + lt * lt / T(S * S));
            const T b = T(1) - sqrt(T(2)) * r;
            wfv = b * b;
        }
        swf[i] = wfv;
    }
    for (int t = threadIdx.x; t < S; t += blockDim.x) {
        T2 v;
        v.x = T(cos_2pi32(t));
        v.y = T(sin_2pi32(t));
        scs[t] = v;
    }
    __syncthreads();

    const T gamma = T(a.gamma);
    const int L = a.L;

    for (long long blk = (long long)blockIdx.x * WARPS + warp; blk < a.nblocks;
         blk += (long long)gridDim.x * WARPS) {
        const int by = (int)(blk / a.nbx);
        const int bx = (int)(blk - (long long)by * a.nbx);
        const int y0 = by * B - L, x0 = bx * B - L;

        // ---- a1/a2: load the support column of this lane and weight it ----
        T zr[S], zi[S];
        const int xc = x0 + lane;
        const bool xin = (unsigned)xc < (unsigned)a.W;
        bool anyk = false;
        unsigned fmax_bits = 0;   // bits of max |f| over known pixels (order-preserving)
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
            const T w = kn ? sw0[m * S + lane] : T(0);
            zr[m] = kn ? T(fv) * w : T(0);   // select: unknown values never enter
            zi[m] = w;
            anyk |= kn;
            const unsigned ab = __float_as_uint(fv) & 0x7fffffffu;
            fmax_bits = (kn && ab > fmax_bits) ? ab : fmax_bits;
        }
        // z = x + j alpha w with alpha = 2^e >= max|f|: both halves of z get the
        // same magnitude, so W keeps full precision through the shared FFT; a
        // power of two is undone exactly.
        fmax_bits = __reduce_max_sync(FULL, fmax_bits);
        unsigned aexp = (fmax_bits >> 23) + 1u;             // exponent field of 2^e
        aexp = (fmax_bits >= 0x00800000u && fmax_bits < 0x7e000000u) ? aexp : 127u;
        const T alpha = T(__uint_as_float(aexp << 23));
        const T inv2alpha = T(__uint_as_float((253u - aexp) << 23));   // 1 / (2 alpha)
#pragma unroll
        for (int m = 0; m < S; ++m) zi[m] = zi[m] * alpha;

        // target pixels of this lane
        int pix_m[P], pix_n[P];
        T gacc[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int pidx = lane + 32 * q;
            pix_m[q] = L + pidx / B;
            pix_n[q] = L + pidx % B;
            gacc[q] = T(0);
        }

        if (__any_sync(FULL, anyk)) {
            // ---- a3: z = x + j w, FFT over m (columns) ----
            fft32<T>(zr, zi);
            // transpose through the (not yet used) W area of this warp
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
            // FFT over n (rows): lane k now holds Z[k][0..31]
            fft32<T>(zr, zi);

            // Separate R_w = F2{x} and W = F2{w}:
            //   R[k][l] = (Z[k][l] + conj Z[-k][-l]) / 2,
            //   W[k][l] = (Z[k][l] - conj Z[-k][-l]) / 2j.
            const int src = (S - lane) & (S - 1);
            T2* wrow_out = Wd + lane * WSTRIDE;
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
                wrow_out[l + S] = w1;
                if (l == 0) W0 = w1.x;
                if (l2 != l) {
                    const T br = zr[l2], bi = zi[l2];
                    T2 w2;
                    w2.x = (bi + di) * inv2alpha;
                    w2.y = (dr - br) * inv2alpha;
                    zr[l2] = (br + dr) * T(0.5);
                    zi[l2] = (bi - di) * T(0.5);
                    wrow_out[l2] = w2;
                    wrow_out[l2 + S] = w2;
                }
            }
            W0 = __shfl_sync(FULL, W0, 0);   // W[0][0] = sum of w

            // frequency weights of this lane's row (w_f[k][l] = w_f[k][S-l])
            T wfr[S / 2 + 1];
#pragma unroll
            for (int l = 0; l <= S / 2; ++l) wfr[l] = swf[lane * S + l];

            T rowmax = T(0);
#pragma unroll
            for (int l = 0; l < S; ++l)
                rowmax = fmax(rowmax, objective<T>(zr[l], zi[l], wfr[l <= S / 2 ? l : S - l]));
            __syncwarp();

            int16_t* seq = a.seq ? a.seq + (size_t)blk * a.K : nullptr;
            for (int nu = 0; nu < a.K; ++nu) {
                // ---- a5: argmax, lowest linear index on ties ----
                const T M = warp_max(rowmax);
                const unsigned cand = __ballot_sync(FULL, rowmax == M);
                const int u = __ffs(cand) - 1;
                if (lane == u) {
#pragma unroll
                    for (int l = 0; l < S; ++l) { T2 v; v.x = zr[l]; v.y = zi[l]; rowbuf[l] = v; }
                }
                __syncwarp();
                const T2 mine = rowbuf[lane];
                const T o = objective<T>(mine.x, mine.y, swf[u * S + lane]);
                const unsigned vb = __ballot_sync(FULL, o == M);
                const int v = __ffs(vb) - 1;
                const T2 Ruv = rowbuf[v];
                __syncwarp();

                // ---- a6: p = R[u,v] / W[0,0]; gamma p enters G (Eq. 11) ----
                const T cr = gamma * (Ruv.x / W0);
                const T ci = gamma * (Ruv.y / W0);
                if (seq != nullptr && lane == 0) seq[nu] = (int16_t)(u * S + v);
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int t = (u * pix_m[q] + v * pix_n[q]) & (S - 1);
                    const T2 cs = scs[t];
                    gacc[q] = fma_rn(cr, cs.x, fma_rn(-ci, cs.y, gacc[q]));
                }

                // ---- a7: R[k,l] -= gamma p W[k-u, l-v], then next objective ----
                const T2* wrow = Wd + ((lane - u) & (S - 1)) * WSTRIDE + ((S - v) & (S - 1));
                rowmax = T(0);
#pragma unroll
                for (int l = 0; l < S; ++l) {
                    const T2 w = wrow[l];
                    zr[l] = fma_rn(-cr, w.x, fma_rn(ci, w.y, zr[l]));
                    zi[l] = fma_rn(-cr, w.y, fma_rn(-ci, w.x, zi[l]));
                    rowmax = fmax(rowmax, objective<T>(zr[l], zi[l], wfr[l <= S / 2 ? l : S - l]));
                }
            }
            __syncwarp();   // W area free for the next block
        } else if (a.seq != nullptr && lane == 0) {
            int16_t* seq = a.seq + (size_t)blk * a.K;
            for (int nu = 0; nu < a.K; ++nu) seq[nu] = -1;
        }

        // ---- a9: write-back of the B x B target ----
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int pidx = lane + 32 * q;
            if (pidx < B * B) {
                const int ty = by * B + pidx / B, tx = bx * B + pidx % B;
                if (ty < a.H && tx < a.W) {
                    const size_t off = (size_t)ty * a.pitch + tx;
                    const bool kn = __ldg(a.mask + off) != 0;
                    a.out[off] = kn ? __ldg(a.img + off) : (float)gacc[q];
                }
            }
        }
    }
}

// Host-side launch helpers (one translation unit per arithmetic type).
struct LaunchInfo {
    int grid;
    int block_threads;
    size_t smem;
};

}  // namespace fsrk
