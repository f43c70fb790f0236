// FSR with a small support S in {8, 16} (Sec. II; the support-size study of
// Sec. IV, Fig. 3): one warp per block, every lane holds P = S*S/32
// consecutive components of the spectrum (row k = lane*P / S, columns
// l0 .. l0+P-1, l0 = lane*P mod S), so the linear index k*S + l of a lane's
// components grows with the lane and with the register index.
//
// The 2-D DFTs of the weighted signal and of the weights (Eq. 7) are two
// direct separable passes through shared memory with a conjugate-symmetric
// twiddle table and one summation order, which makes R_w and W exactly
// Hermitian (the ties of the first iteration are exact, as in the oracle).
// The iteration follows the S = 32 kernel: the weighted mean mu is removed
// (R_w = mu W + Q), the DC phase keeps R = a W + Q, the objective of Eq. (8)
// is rounded explicitly, the argmax takes the lowest linear index on ties,
// the residual update of Eq. (12) reads W rows stored with their first P
// entries repeated (no index wrap), and Re g is accumulated at the B x B
// target pixels only.  Work comes from the same work table and counter as
// the S = 32 batch kernel.
#include "fsr_launch.h"

namespace fsrk {
namespace {

constexpr int kWarpsSmall = 8;

template <typename T, int SZ>
struct SmallLayout {
    using T2 = typename Vec2<T>::type;
    static constexpr int SS = SZ * SZ;
    static constexpr int P = SS / 32;              // components per lane
    // Row strides with padding against bank conflicts: the lanes of a
    // half-warp touch 8 (S = 16) or 4 (S = 8) different rows at once.
    static constexpr int XS = SZ + 1;              // x, w of the support (T)
    static constexpr int YS = SZ + 1;              // first-pass outputs (T2)
    static constexpr int WROW = 2 * SZ + 1;        // W row: its S entries, the first P again, pad
    // CTA tables: w0, w_f (SS T each), e^{-j 2 pi t / S} (S T2)
    static constexpr size_t w0_off = 0;
    static constexpr size_t wf_off = w0_off + sizeof(T) * SS;
    static constexpr size_t tw_off = wf_off + sizeof(T) * SS;
    static constexpr size_t warp0_off = (tw_off + sizeof(T2) * SZ + 127) & ~(size_t)127;
    // per warp: region A = x and w of the support (prologue), then the W rows;
    // region B = the first-pass outputs Yx, Yw
    static constexpr size_t a_bytes = sizeof(T2) * SZ * WROW > 2 * sizeof(T) * SZ * XS ? sizeof(T2) * SZ * WROW
                                                                                       : 2 * sizeof(T) * SZ * XS;
    static constexpr size_t b_bytes = 2 * sizeof(T2) * SZ * YS;
    static constexpr size_t per_warp = (a_bytes + b_bytes + 127) & ~(size_t)127;
    static constexpr size_t bytes(int warps) { return warp0_off + per_warp * (size_t)warps; }
};

template <typename T, int SZ>
__device__ __forceinline__ void small_tables(const MethodArgs& mth, T* sw0, T* swf, typename Vec2<T>::type* stw) {
    const T half = T(SZ) / T(2);
    for (int i = threadIdx.x; i < SZ * SZ; i += blockDim.x) {
        const int m = i / SZ, n = i % SZ;
        const T dm = T(m) - T(SZ - 1) / T(2), dn = T(n) - T(SZ - 1) / T(2);
        sw0[i] = pow(T(mth.rho), sqrt(dm * dm + dn * dn));
        T wfv = T(1);
        if (mth.freq_weight) {
            const T kt = half - fabs(T(m) - half), lt = half - fabs(T(n) - half);
            const T r = sqrt(kt * kt / T(SZ * SZ) + lt * lt / T(SZ * SZ));
            const T b = T(1) - sqrt(T(2)) * r;
            wfv = b * b;
        }
        swf[i] = wfv;
    }
    for (int t = threadIdx.x; t < SZ; t += blockDim.x) {
        typename Vec2<T>::type v;
        v.x = T(cos_2pi32(t * (32 / SZ)));
        v.y = T(-sin_2pi32(t * (32 / SZ)));   // e^{-j 2 pi t / S}
        stw[t] = v;
    }
}

// One block: a1-a9 for support size SZ, target B x B.
template <typename T, int SZ, int B>
__device__ __forceinline__ void small_block(const ImageArgs& im, long long blk, int L, T gamma, const T* sw0,
                                            const T* swf, const typename Vec2<T>::type* stw, unsigned char* area,
                                            unsigned long long* empty, int lane) {
    using T2 = typename Vec2<T>::type;
    using Lay = SmallLayout<T, SZ>;
    constexpr int P = Lay::P, WROW = Lay::WROW, XS = Lay::XS, YS = Lay::YS;
    constexpr int PT = TargetPix<B>::P;
    T* xs = reinterpret_cast<T*>(area);                 // region A (prologue)
    T* ws = xs + SZ * XS;
    T2* Wr = reinterpret_cast<T2*>(area);               // region A (after pass 1)
    T2* Yx = reinterpret_cast<T2*>(area + Lay::a_bytes);
    T2* Yw = Yx + SZ * YS;

    const int by = (int)(blk / im.nbx);
    const int bx = (int)(blk - (long long)by * im.nbx);
    const int y0 = by * B - L, x0 = bx * B - L;
    const int k = (lane * P) / SZ, l0 = (lane * P) % SZ;   // this lane's row and first column
    int16_t* seq = im.seq ? im.seq + (size_t)blk * im.K : nullptr;

    // ---- a1, a2: load the support, weights, weighted mean ----
    __syncwarp();   // the area is free (previous block done)
    T sw = T(0), sfw = T(0);
    unsigned anyk = 0;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int i = lane + 32 * j;
        const int m = i / SZ, n = i % SZ;
        const int y = y0 + m, x = x0 + n;
        bool kn = false;
        float fv = 0.f;
        if ((unsigned)y < (unsigned)im.H && (unsigned)x < (unsigned)im.W) {
            const size_t off = (size_t)y * im.pitch + x;
            kn = __ldg(im.mask + off) != 0;
            fv = __ldg(im.img + off);
        }
        const T f = kn ? T(fv) : T(0);   // select: unknown values never enter arithmetic
        const T w = kn ? sw0[i] : T(0);
        xs[m * XS + n] = f;
        ws[m * XS + n] = w;
        sw += w;
        sfw += w * f;
        anyk |= kn ? 1u : 0u;
    }
    T gacc[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) gacc[q] = T(0);

    if (__ballot_sync(FULL, anyk != 0) != 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sw += __shfl_xor_sync(FULL, sw, o);
            sfw += __shfl_xor_sync(FULL, sfw, o);
        }
        const T mu = sfw / sw;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int i = lane + 32 * j;
            const int x = (i / SZ) * XS + i % SZ;
            xs[x] = ws[x] > T(0) ? (xs[x] - mu) * ws[x] : T(0);
        }
        __syncwarp();

        // ---- a3, pass 1 (over n): Y[m][l] = sum_n v[m][n] e^{-j 2 pi l n / S} ----
        {
            T xr[SZ], wr_[SZ];
#pragma unroll
            for (int n = 0; n < SZ; ++n) {
                xr[n] = xs[k * XS + n];
                wr_[n] = ws[k * XS + n];
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const int l = l0 + p;
                T axr = T(0), axi = T(0), awr = T(0), awi = T(0);
#pragma unroll
                for (int n = 0; n < SZ; ++n) {
                    const T2 t = stw[(l * n) & (SZ - 1)];
                    axr = fma_rn(xr[n], t.x, axr);
                    axi = fma_rn(xr[n], t.y, axi);
                    awr = fma_rn(wr_[n], t.x, awr);
                    awi = fma_rn(wr_[n], t.y, awi);
                }
                T2 vx, vw;
                vx.x = axr; vx.y = axi;
                vw.x = awr; vw.y = awi;
                Yx[k * YS + l] = vx;   // row m = k of this lane
                Yw[k * YS + l] = vw;
            }
        }
        __syncwarp();

        // ---- a3, pass 2 (over m): Z[k][l] = sum_m Y[m][l] e^{-j 2 pi k m / S} ----
        T zr[P], zi[P], w0r = T(0);
        {
            T2 wv[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                zr[p] = zi[p] = T(0);
                wv[p].x = wv[p].y = T(0);
            }
#pragma unroll
            for (int m = 0; m < SZ; ++m) {
                const T2 t = stw[(k * m) & (SZ - 1)];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const T2 a = Yx[m * YS + l0 + p];
                    const T2 b = Yw[m * YS + l0 + p];
                    zr[p] = fma_rn(a.x, t.x, fma_rn(-a.y, t.y, zr[p]));
                    zi[p] = fma_rn(a.x, t.y, fma_rn(a.y, t.x, zi[p]));
                    wv[p].x = fma_rn(b.x, t.x, fma_rn(-b.y, t.y, wv[p].x));
                    wv[p].y = fma_rn(b.x, t.y, fma_rn(b.y, t.x, wv[p].y));
                }
            }
            __syncwarp();   // region A (x, w) is read no more: W rows go there
#pragma unroll
            for (int p = 0; p < P; ++p) {
                Wr[k * WROW + l0 + p] = wv[p];
                if (l0 + p < P) Wr[k * WROW + SZ + l0 + p] = wv[p];
            }
            if (lane == 0) w0r = wv[0].x;   // W[0][0] (component 0 of lane 0)
        }
        const T W0 = __shfl_sync(FULL, w0r, 0);
        __syncwarp();

        // ---- a4-a8 ----
        T wfv[P];
#pragma unroll
        for (int p = 0; p < P; ++p) wfv[p] = swf[k * SZ + l0 + p];
        int pm[PT], pn[PT];
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            pm[q] = L + (lane + 32 * q) / B;
            pn[q] = L + (lane + 32 * q) % B;
        }
        const T invW0 = T(1) / W0;
        T o[P];
        int nu = 0;
        T cr = T(0), ci = T(0);
        int u = 0, v = 0;

        // a5 for the objectives o[] of this lane's components with values
        // (vr, vi): block maximum, lowest lane holding it, its first
        // component; a6: c, the recorded index, the target pixels.
        auto pick = [&](const T (&vr)[P], const T (&vi)[P]) {
            T mx;
            if constexpr (sizeof(T) == 4 && P == 8) {
                mx = max3(max3(o[0], o[1], o[2]), max3(o[3], o[4], o[5]), fmaxf(o[6], o[7]));
            } else if constexpr (sizeof(T) == 4) {
                mx = o[0];
#pragma unroll
                for (int p = 1; p < P; ++p) mx = fmaxf(mx, o[p]);
            } else {
                mx = o[0];
#pragma unroll
                for (int p = 1; p < P; ++p) mx = fmax(mx, o[p]);
            }
            T Mx = mx;
            if constexpr (sizeof(T) == 4) {
                // objective values are >= +0: their bit patterns order like the values
                Mx = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(float(mx))));
            } else {
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) {
                    const T oth = __shfl_xor_sync(FULL, Mx, s);
                    Mx = oth > Mx ? oth : Mx;
                }
            }
            const int ul = __ffs(__ballot_sync(FULL, mx == Mx)) - 1;
            int pf = P - 1;
            T sr = vr[P - 1], si = vi[P - 1];
#pragma unroll
            for (int p = P - 2; p >= 0; --p) {
                const bool hit = o[p] == Mx;
                pf = hit ? p : pf;
                sr = hit ? vr[p] : sr;
                si = hit ? vi[p] : si;
            }
            pf = __shfl_sync(FULL, pf, ul);
            const T Rr = __shfl_sync(FULL, sr, ul);
            const T Ri = __shfl_sync(FULL, si, ul);
            const int c = ul * P + pf;
            u = c / SZ;
            v = c % SZ;
            cr = gamma * (Rr * invW0);
            ci = gamma * (Ri * invW0);
            if (seq != nullptr && lane == 0) seq[nu] = (int16_t)(u * SZ + v);
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const T2 e = stw[(SZ - ((u * pm[q] + v * pn[q]) & (SZ - 1))) & (SZ - 1)];   // e^{+j...}
                gacc[q] = fma_rn(cr, e.x, fma_rn(-ci, e.y, gacc[q]));   // Re(c e^{+j theta})
            }
        };

        // ---- DC phase: R = a W + Q ----
        bool done = im.K <= 0;
        if (!done) {
            T ar = mu, ai = T(0);
            for (;;) {
                T rr[P], ri[P];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const T2 w = Wr[k * WROW + l0 + p];
                    split_value(ar, ai, w.x, w.y, zr[p], zi[p], rr[p], ri[p]);
                    o[p] = objective<T>(rr[p], ri[p], wfv[p]);
                }
                pick(rr, ri);
                if (++nu == im.K) {
                    done = true;
                    break;
                }
                if ((u | v) != 0) break;
                ar -= cr;
                ai -= ci;
            }
            if (!done) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const T2 w = Wr[k * WROW + l0 + p];
                    split_value(ar, ai, w.x, w.y, zr[p], zi[p], zr[p], zi[p]);
                }
            }
        }
        // ---- a7 (Eq. 12) for the last pick and the next objective, a5-a6 ----
        while (!done) {
            const T2* row = Wr + ((k - u) & (SZ - 1)) * WROW + ((l0 - v) & (SZ - 1));
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const T2 w = row[p];
                residual_update(zr[p], zi[p], w.x, w.y, cr, ci);
                o[p] = objective<T>(zr[p], zi[p], wfv[p]);
            }
            pick(zr, zi);
            if (++nu == im.K) done = true;
        }
    } else if (lane == 0) {
        empty_block(seq, im.K, empty);
    }

    // ---- a9: write-back of the B x B target ----
#pragma unroll
    for (int q = 0; q < PT; ++q) {
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
}

template <typename T, int SZ, int B, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) fsr_small_kernel(const BatchArgs a) {
    using Lay = SmallLayout<T, SZ>;
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    T* sw0 = reinterpret_cast<T*>(smem + Lay::w0_off);
    T* swf = reinterpret_cast<T*>(smem + Lay::wf_off);
    T2* stw = reinterpret_cast<T2*>(smem + Lay::tw_off);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char* area = smem + Lay::warp0_off + Lay::per_warp * warp;
    small_tables<T, SZ>(a.mth, sw0, swf, stw);
    __syncthreads();

    const T gamma = T(a.mth.gamma);
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.counter, (unsigned long long)a.chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= (unsigned long long)a.total) break;
        const long long end = min((long long)base + a.chunk, a.total);
        for (long long item = (long long)base; item < end; ++item) {
            int lo = 0, hi = a.n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(a.first + mid) <= item) lo = mid;
                else hi = mid - 1;
            }
            const ImageArgs im = a.images[lo];
            small_block<T, SZ, B>(im, item - __ldg(a.first + lo), a.mth.L, gamma, sw0, swf, stw, area, a.empty,
                                  lane);
        }
    }
}

template <typename T, int SZ, int B>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(fsr_small_kernel<T, SZ, B, kWarpsSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SmallLayout<T, SZ>::bytes(kWarpsSmall));
}

template <typename T, int SZ, int B>
cudaError_t launch_one(const BatchArgs& a, int chunk, int sm_count, cudaStream_t stream) {
    const size_t smem = SmallLayout<T, SZ>::bytes(kWarpsSmall);
    int grid = 0;
    cudaError_t e = persistent_grid(fsr_small_kernel<T, SZ, B, kWarpsSmall>, kWarpsSmall, smem,
                                    (a.total + chunk - 1) / chunk, sm_count, &grid);
    if (e != cudaSuccess) return e;
    fsr_small_kernel<T, SZ, B, kWarpsSmall><<<grid, kWarpsSmall * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t configure_all() {
    cudaError_t e;
    if ((e = configure_one<T, 16, 2>()) != cudaSuccess) return e;
    if ((e = configure_one<T, 16, 4>()) != cudaSuccess) return e;
    if ((e = configure_one<T, 16, 8>()) != cudaSuccess) return e;
    if ((e = configure_one<T, 8, 2>()) != cudaSuccess) return e;
    return configure_one<T, 8, 4>();
}

template <typename T>
cudaError_t launch_any(const BatchArgs& a, int S, int B, int chunk, int sm_count, cudaStream_t stream) {
    if (S == 16 && B == 2) return launch_one<T, 16, 2>(a, chunk, sm_count, stream);
    if (S == 16 && B == 4) return launch_one<T, 16, 4>(a, chunk, sm_count, stream);
    if (S == 16 && B == 8) return launch_one<T, 16, 8>(a, chunk, sm_count, stream);
    if (S == 8 && B == 2) return launch_one<T, 8, 2>(a, chunk, sm_count, stream);
    if (S == 8 && B == 4) return launch_one<T, 8, 4>(a, chunk, sm_count, stream);
    return cudaErrorNotSupported;
}

}  // namespace

bool small_supported(int S, int B) { return (S == 16 && (B == 2 || B == 4 || B == 8)) || (S == 8 && (B == 2 || B == 4)); }

cudaError_t configure_small() {
    cudaError_t e = configure_all<float>();
    if (e != cudaSuccess) return e;
    return configure_all<double>();
}

cudaError_t launch_batch_small(const BatchArgs& a, int S, int B, int fp64, int chunk, int sm_count,
                               cudaStream_t stream) {
    return fp64 ? launch_any<double>(a, S, B, chunk, sm_count, stream)
                : launch_any<float>(a, S, B, chunk, sm_count, stream);
}

}  // namespace fsrk
