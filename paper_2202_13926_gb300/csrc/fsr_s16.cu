// FP32 FSR with the 16 x 16 support (B in {2, 4, 8}; the support of the
// paper's frame-rate study, Sec. IV, Fig. 5): one half-warp per block, two
// blocks per warp.  Lane t of a half holds column t of the support, then row
// t of the spectrum (16 complex values in registers), as the S = 32 kernel
// does with a whole warp:
//   a1-a3  the support is loaded by columns, the weighted mean mu is removed,
//          x = (f - mu) w and alpha w are packed into z = x + j alpha w, and
//          the 2-D DFT of Eq. (7) is two in-register radix-2 FFTs of length
//          16 with a transpose through shared memory; R_w and W are formed
//          from Z[k][l] and conj Z[-k][-l] with commutative operations, so
//          both are exactly Hermitian (the ties of the first iteration are
//          exact, as in the oracle);
//   a4-a8  R = a W + Q while only the DC component is selected (DC phase),
//          then Q alone; Eq. (12) reads the shifted W row of 31 stored
//          entries (the first 15 repeated: no column wrap) with 8-byte loads,
//          free of bank conflicts with rows of 33 entries; the objective of
//          Eq. (8) is rounded explicitly; the lane holding the block maximum
//          publishes its row in shared memory and lane t of the half forms
//          the objective of component t again, so the lowest index with the
//          maximum is found by two ballots;
//   a9     Re g (sparse inverse of G) accumulated at the target pixels only.
// The two blocks of a warp may have different K and leave the DC phase at
// different iterations: the loop runs to the larger K and every step that is
// specific to one half is plain arithmetic on its lanes; every shuffle,
// ballot and warp barrier is reached by all 32 lanes.
#include "fsr_launch.h"

namespace fsrk {
namespace {

constexpr int S16 = 16;
constexpr int WS16 = 33;    // W row stride (float2): 16 entries, the first 15 again, pad
constexpr int TS16 = 17;    // transpose stride (float2)
constexpr int WFS16 = 17;   // w_f row stride (float)
constexpr int kWarpsS16 = 8;
constexpr unsigned kBlockBytes = S16 * WS16 * 8 + S16 * 8;   // W rows (also the transpose), published row
static_assert(S16 * TS16 <= S16 * WS16, "the transpose fits in the W area");
static_assert((S16 * WS16 * 8) % 16 == 0, "the published row is 16-byte aligned");

constexpr size_t kW0Off = 0;                                   // w0[m][n], S x S
constexpr size_t kWfOff = kW0Off + 4 * S16 * S16;              // w_f[k][l], S x WFS16
constexpr size_t kCsOff = kWfOff + 4 * S16 * WFS16;            // (cos, sin)(2 pi t / S)
constexpr size_t kWarp0Off = (kCsOff + 8 * S16 + 127) & ~(size_t)127;
constexpr size_t kPerWarp = 2 * (size_t)kBlockBytes;
constexpr size_t smem_bytes(int warps) { return kWarp0Off + kPerWarp * (size_t)warps; }

__host__ __device__ constexpr int brev4(int i) { return ((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3); }

// In-register radix-2 decimation-in-time FFT of length 16, natural order in
// and out, X[k] = sum_m x[m] e^{-j 2 pi k m / 16}.
__device__ __forceinline__ void fft16(float (&re)[S16], float (&im)[S16]) {
    float ar[S16], ai[S16];
#pragma unroll
    for (int i = 0; i < S16; ++i) {
        ar[i] = re[brev4(i)];
        ai[i] = im[brev4(i)];
    }
#pragma unroll
    for (int half = 1; half < S16; half *= 2) {
#pragma unroll
        for (int j = 0; j < S16; j += 2 * half) {
#pragma unroll
            for (int t = 0; t < half; ++t) {
                const int tw = t * (8 / half);   // e^{-j 2 pi tw / 16}
                const float br = ar[j + t + half], bi = ai[j + t + half];
                float xr, xi;
                if (tw == 0) {
                    xr = br;
                    xi = bi;
                } else if (tw == 4) {   // times -j
                    xr = bi;
                    xi = -br;
                } else {
                    const float c = float(cos_2pi32(2 * tw)), s = float(-sin_2pi32(2 * tw));
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
    for (int i = 0; i < S16; ++i) {
        re[i] = ar[i];
        im[i] = ai[i];
    }
}

// butterfly maximum of nonnegative-float bit patterns within a half-warp
__device__ __forceinline__ unsigned half_max(unsigned v) {
#pragma unroll
    for (int s = 8; s > 0; s >>= 1) v = max(v, (unsigned)__shfl_xor_sync(FULL, v, s));
    return v;
}
__device__ __forceinline__ float half_sum(float v) {
#pragma unroll
    for (int s = 8; s > 0; s >>= 1) v += __shfl_xor_sync(FULL, v, s);
    return v;
}

__device__ __forceinline__ float wf16(const float (&wfr)[S16 / 2 + 1], int l) {
    return wfr[l <= S16 / 2 ? l : S16 - l];
}

// maximum of the objective over the lane's row of R = a W + Q (unshifted W row)
__device__ __forceinline__ float split_objective_row(const float (&zr)[S16], const float (&zi)[S16],
                                                     const float (&wfr)[S16 / 2 + 1], const float2* wrow, float ar,
                                                     float ai) {
    float o[S16];
#pragma unroll
    for (int l = 0; l < S16; ++l) {
        const float2 w = wrow[l];
        float rr, ri;
        split_value(ar, ai, w.x, w.y, zr[l], zi[l], rr, ri);
        o[l] = objective<float>(rr, ri, wf16(wfr, l));
    }
    float m = fmaxf(o[0], o[1]);
#pragma unroll
    for (int l = 2; l < S16; l += 2) m = max3(m, o[l], o[l + 1]);
    return m;
}

template <int B>
__device__ __forceinline__ void block16(const ImageArgs& im, long long blk, bool valid, int Kmax, int L, float gamma,
                                        const float* __restrict__ sw0, const float* __restrict__ swf,
                                        const float2* __restrict__ scs, float2* Wd, float2* rowbuf,
                                        unsigned long long* empty, int lane) {
    constexpr int PT = (B * B + S16 - 1) / S16;   // target pixels per lane
    const int t = lane & 15, hb = lane & 16;
    int by = 0, bx = 0;
    if (valid) {
        by = (int)(blk / im.nbx);
        bx = (int)(blk - (long long)by * im.nbx);
    }
    const int y0 = by * B - L, x0 = bx * B - L;

    // ---- a1, a2: column t of the support, weights, weighted mean ----
    float zr[S16], zi[S16];
    unsigned known = 0;
    const int x = x0 + t;
#pragma unroll
    for (int m = 0; m < S16; ++m) {
        const int y = y0 + m;
        float f = 0.f;
        if (valid && (unsigned)y < (unsigned)im.H && (unsigned)x < (unsigned)im.W) {
            const size_t off = (size_t)y * im.pitch + x;
            if (__ldg(im.mask + off) != 0) {
                known |= 1u << m;
                f = __ldg(im.img + off);
            }
        }
        zr[m] = f;   // unknown values never enter arithmetic
    }
    float sw = 0.f, sfw = 0.f;
#pragma unroll
    for (int m = 0; m < S16; ++m) {
        const float w = ((known >> m) & 1u) ? sw0[m * S16 + t] : 0.f;
        sw += w;
        sfw += w * zr[m];
    }
    sw = half_sum(sw);
    sfw = half_sum(sfw);
    const unsigned kb = (__ballot_sync(FULL, known != 0) >> hb) & 0xFFFFu;
    const bool active = valid && kb != 0u;
    const float mu = active ? sfw / sw : 0.f;
    unsigned dmax = 0;
#pragma unroll
    for (int m = 0; m < S16; ++m) {
        const bool kn = (known >> m) & 1u;
        const float w = kn ? sw0[m * S16 + t] : 0.f;
        const float d = zr[m] - mu;
        zr[m] = kn ? d * w : 0.f;
        zi[m] = w;
        const unsigned ab = __float_as_uint(d) & 0x7fffffffu;
        dmax = (kn && ab > dmax) ? ab : dmax;
    }
    // alpha = 2^e >= max |f - mu|: both halves of z = x + j alpha w have one
    // magnitude through the shared FFT; powers of two are undone exactly
    dmax = half_max(dmax);
    unsigned aexp = (dmax >> 23) + 1u;
    aexp = (dmax >= 0x00800000u && dmax < 0x7e000000u) ? aexp : 127u;
    const float alpha = __uint_as_float(aexp << 23);
    const float inv2alpha = __uint_as_float((253u - aexp) << 23);
#pragma unroll
    for (int m = 0; m < S16; ++m) zi[m] *= alpha;

    // ---- a3: FFT over m (lane t holds column t), transpose, FFT over n ----
    fft16(zr, zi);
    __syncwarp();   // the W area of the previous blocks is free
#pragma unroll
    for (int k = 0; k < S16; ++k) Wd[k * TS16 + t] = make_float2(zr[k], zi[k]);
    __syncwarp();
#pragma unroll
    for (int n = 0; n < S16; ++n) {
        const float2 v = Wd[t * TS16 + n];
        zr[n] = v.x;
        zi[n] = v.y;
    }
    __syncwarp();
    fft16(zr, zi);   // lane k = t holds Z[k][0..15]

    // Q[k][l] = (Z[k][l] + conj Z[-k][-l]) / 2,  W[k][l] = (Z[k][l] - conj Z[-k][-l]) / (2j alpha)
    const int src = hb + ((S16 - t) & (S16 - 1));
    float2* wrow_out = Wd + t * WS16;
    float w00 = 0.f;
#pragma unroll
    for (int l = 0; l <= S16 / 2; ++l) {
        const int l2 = (S16 - l) & (S16 - 1);
        const float cr = __shfl_sync(FULL, zr[l2], src);
        const float ci = __shfl_sync(FULL, zi[l2], src);
        float dr = cr, di = ci;
        if (l2 != l) {
            dr = __shfl_sync(FULL, zr[l], src);
            di = __shfl_sync(FULL, zi[l], src);
        }
        const float ar = zr[l], ai = zi[l];
        const float2 w1 = make_float2((ai + ci) * inv2alpha, (cr - ar) * inv2alpha);
        zr[l] = (ar + cr) * 0.5f;
        zi[l] = (ai - ci) * 0.5f;
        wrow_out[l] = w1;
        if (l < S16 - 1) wrow_out[l + S16] = w1;
        if (l == 0) w00 = w1.x;
        if (l2 != l) {
            const float br = zr[l2], bi = zi[l2];
            const float2 w2 = make_float2((bi + di) * inv2alpha, (dr - br) * inv2alpha);
            zr[l2] = (br + dr) * 0.5f;
            zi[l2] = (bi - di) * 0.5f;
            wrow_out[l2] = w2;
            if (l2 < S16 - 1) wrow_out[l2 + S16] = w2;
        }
    }
    const float W0 = __shfl_sync(FULL, w00, hb);
    __syncwarp();

    // ---- a4-a8 ----
    float wfr[S16 / 2 + 1];
#pragma unroll
    for (int l = 0; l <= S16 / 2; ++l) wfr[l] = swf[t * WFS16 + l];
    int pm[PT], pn[PT];
    float gacc[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        pm[q] = L + (t + S16 * q) / B;
        pn[q] = L + (t + S16 * q) % B;
        gacc[q] = 0.f;
    }
    const int Kh = valid ? im.K : 0;
    int16_t* seq = (valid && im.seq) ? im.seq + (size_t)blk * im.K : nullptr;
    if (valid && !active && t == 0) empty_block(seq, im.K, empty);
    const float invW0 = active ? 1.f / W0 : 0.f;
    bool split = true;             // R = a W + Q (DC phase)
    float ar = mu, ai = 0.f;
    float m_lane = (active && Kh > 0) ? split_objective_row(zr, zi, wfr, Wd + t * WS16, ar, ai) : 0.f;

    for (int nu = 0; nu < Kmax; ++nu) {   // uniform over the warp
        const bool run = active && nu < Kh;
        // a5: block maximum (each half reduces over its own 16 lanes), the
        // lowest row holding it, then its lowest column
        const unsigned Mb = __reduce_max_sync(0xFFFFu << hb, run ? __float_as_uint(m_lane) : 0u);
        const unsigned ub = (__ballot_sync(FULL, run && __float_as_uint(m_lane) == Mb) >> hb) & 0xFFFFu;
        const int u = ub ? __ffs(ub) - 1 : 0;
        __syncwarp();   // the previous pick's reads of the published row are done
        if (run && t == u) {
            float4* pub = reinterpret_cast<float4*>(rowbuf);
#pragma unroll
            for (int i = 0; i < S16 / 2; ++i) pub[i] = make_float4(zr[2 * i], zi[2 * i], zr[2 * i + 1], zi[2 * i + 1]);
        }
        __syncwarp();
        const float2 qv = rowbuf[t];
        float rr = qv.x, ri = qv.y;
        if (split) {
            const float2 w = Wd[u * WS16 + t];
            split_value(ar, ai, w.x, w.y, qv.x, qv.y, rr, ri);
        }
        const float o = objective<float>(rr, ri, swf[u * WFS16 + t]);
        const unsigned vbits = (__ballot_sync(FULL, run && __float_as_uint(o) == Mb) >> hb) & 0xFFFFu;
        const int v = vbits ? __ffs(vbits) - 1 : 0;
        const float Rr = __shfl_sync(FULL, rr, hb + v);
        const float Ri = __shfl_sync(FULL, ri, hb + v);

        // a6 (Eqs. 10, 11): c = gamma p, the target pixels of the sparse inverse
        const float cr = gamma * (Rr * invW0), ci = gamma * (Ri * invW0);
        if (run) {
            if (seq != nullptr && t == 0) seq[nu] = (int16_t)(u * S16 + v);
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const float2 cs = scs[(u * pm[q] + v * pn[q]) & (S16 - 1)];
                gacc[q] = fma_rn(cr, cs.x, fma_rn(-ci, cs.y, gacc[q]));
            }
        }
        // a7 (Eq. 12) and the objective of the next iteration (this half only)
        if (run && nu + 1 < Kh) {
            if (split && (u | v) == 0) {
                ar -= cr;
                ai -= ci;
                m_lane = split_objective_row(zr, zi, wfr, Wd + t * WS16, ar, ai);
            } else {
                if (split) {   // fold a W into Q
                    const float2* wk = Wd + t * WS16;
#pragma unroll
                    for (int l = 0; l < S16; ++l) {
                        const float2 w = wk[l];
                        split_value(ar, ai, w.x, w.y, zr[l], zi[l], zr[l], zi[l]);
                    }
                    split = false;
                }
                const float2* row = Wd + ((t - u) & (S16 - 1)) * WS16 + ((S16 - v) & (S16 - 1));
                float o2[S16];
#pragma unroll
                for (int l = 0; l < S16; ++l) {
                    const float2 w = row[l];
                    residual_update(zr[l], zi[l], w.x, w.y, cr, ci);
                    o2[l] = objective<float>(zr[l], zi[l], wf16(wfr, l));
                }
                float mm = fmaxf(o2[0], o2[1]);
#pragma unroll
                for (int l = 2; l < S16; l += 2) mm = max3(mm, o2[l], o2[l + 1]);
                m_lane = mm;
            }
        }
    }

    // ---- a9: write-back of the B x B target ----
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int pidx = t + S16 * q;
        if (valid && pidx < B * B) {
            const int ty = by * B + pidx / B, tx = bx * B + pidx % B;
            if (ty < im.H && tx < im.W) {
                const size_t off = (size_t)ty * im.pitch + tx;
                const bool kn = __ldg(im.mask + off) != 0;
                im.out[off] = kn ? __ldg(im.img + off) : gacc[q];
            }
        }
    }
}

template <int B, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 16 / WARPS) fsr_s16_kernel(const BatchArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* sw0 = reinterpret_cast<float*>(smem + kW0Off);
    float* swf = reinterpret_cast<float*>(smem + kWfOff);
    float2* scs = reinterpret_cast<float2*>(smem + kCsOff);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int half = lane >> 4;
    float2* Wd = reinterpret_cast<float2*>(smem + kWarp0Off + kPerWarp * warp + (size_t)kBlockBytes * half);
    float2* rowbuf = Wd + S16 * WS16;

    // tables: Eq. (5) without the known-set factor, Eq. (9), cos/sin(2 pi t / S)
    const float hs = float(S16) / 2.f;
    for (int i = threadIdx.x; i < S16 * S16; i += blockDim.x) {
        const int m = i / S16, n = i % S16;
        const float dm = float(m) - float(S16 - 1) / 2.f, dn = float(n) - float(S16 - 1) / 2.f;
        sw0[i] = powf(a.mth.rho, sqrtf(dm * dm + dn * dn));
        float wfv = 1.f;
        if (a.mth.freq_weight) {
            const float kt = hs - fabsf(float(m) - hs), lt = hs - fabsf(float(n) - hs);
            const float r = sqrtf(kt * kt / float(S16 * S16) + lt * lt / float(S16 * S16));
            const float b = 1.f - sqrtf(2.f) * r;
            wfv = b * b;
        }
        swf[m * WFS16 + n] = wfv;
    }
    for (int i = threadIdx.x; i < S16; i += blockDim.x)
        scs[i] = make_float2(float(cos_2pi32(2 * i)), float(sin_2pi32(2 * i)));
    __syncthreads();

    const float gamma = a.mth.gamma;
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
            block16<B>(im, blk, valid, Kmax, a.mth.L, gamma, sw0, swf, scs, Wd, rowbuf, a.empty, lane);
        }
    }
}

template <int B>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(fsr_s16_kernel<B, kWarpsS16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes(kWarpsS16));
}

template <int B>
cudaError_t launch_one(const BatchArgs& a, int chunk, int sm_count, cudaStream_t stream) {
    const size_t smem = smem_bytes(kWarpsS16);
    int grid = 0;
    cudaError_t e = persistent_grid(fsr_s16_kernel<B, kWarpsS16>, kWarpsS16, smem, (a.total + 2ll * chunk - 1) / (2ll * chunk),
                        sm_count, &grid);
    if (e != cudaSuccess) return e;
    fsr_s16_kernel<B, kWarpsS16><<<grid, kWarpsS16 * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_s16() {
    cudaError_t e;
    if ((e = configure_one<2>()) != cudaSuccess) return e;
    if ((e = configure_one<4>()) != cudaSuccess) return e;
    return configure_one<8>();
}

cudaError_t launch_s16(const BatchArgs& a, int B, int chunk, int sm_count, cudaStream_t stream) {
    switch (B) {
        case 2: return launch_one<2>(a, chunk, sm_count, stream);
        case 4: return launch_one<4>(a, chunk, sm_count, stream);
        case 8: return launch_one<8>(a, chunk, sm_count, stream);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace fsrk
