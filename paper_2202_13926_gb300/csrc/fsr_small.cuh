// FSR with a support S in {8, 16, 24} (Sec. II; the support-size study of
// Sec. IV, Fig. 3): one warp per block.  Every lane holds a patch of RP rows
// x CP columns of the spectrum (P = RP * CP = S*S/32 components; lane
// a * (S/CP) + b holds rows a*RP .. a*RP+RP-1 and columns b*CP .. b*CP+CP-1),
// in registers in row-major order.  For S = 8 and 16 a patch is one row
// segment (RP = 1), so the linear index k*S + l of a lane's components grows
// with the lane and with the register index; for S = 24 (RP = 6, CP = 3) the
// lowest linear index among the maxima is found by a second warp reduction.
// The 6 x 3 patches with W rows of 28 entries make the shifted W reads of
// Eq. (12) free of bank conflicts for every (u, v): the eight column starts
// 3b - v of a half-warp are distinct mod 8 and its two row groups are 6 rows
// = 8 banks apart.
//
// The 2-D DFTs of the weighted signal and of the weights (Eq. 7) are two
// direct separable passes through shared memory with a conjugate-symmetric
// twiddle table and one summation order, which makes R_w and W exactly
// Hermitian (the ties of the first iteration are exact, as in the oracle).
// The iteration follows the S = 32 kernel: the weighted mean mu is removed
// (R_w = mu W + Q), the DC phase keeps R = a W + Q, the objective of Eq. (8)
// is rounded explicitly, the argmax takes the lowest linear index on ties,
// the residual update of Eq. (12) reads W rows stored with their first
// columns repeated (no column wrap), and Re g is accumulated at the B x B
// target pixels only.  Work comes from the same work table and counter as
// the S = 32 batch kernel.
#pragma once

#include "fsr_launch.h"

namespace fsrk {
namespace small {

// cos(pi t / 12) for t = 0..6 (mathematical constants).
__host__ __device__ constexpr double cos_pi12_base(int t) {
    return t == 0 ? 1.0
         : t == 1 ? 0.965925826289068286749743199728897367
         : t == 2 ? 0.866025403784438646763723170752936183
         : t == 3 ? 0.707106781186547524400844362104849039
         : t == 4 ? 0.5
         : t == 5 ? 0.258819045102520762348898837624048328
         : 0.0;
}
// cos(2 pi t / 24) for any integer t, exact on the axes and at pi/3.
__host__ __device__ constexpr double cos_2pi24(int t) {
    t %= 24;
    if (t < 0) t += 24;
    return t <= 6 ? cos_pi12_base(t)
         : t <= 12 ? -cos_pi12_base(12 - t)
         : t <= 18 ? -cos_pi12_base(t - 12)
         : cos_pi12_base(24 - t);
}
// cos and sin of 2 pi t / S for S in {8, 16, 24, 32}; cos(S - t) = cos(t) and
// sin(S - t) = -sin(t) hold bit for bit.
template <int SZ>
__host__ __device__ constexpr double cos_2pi(int t) {
    if constexpr (SZ == 24) return cos_2pi24(t);
    else return cos_2pi32(t * (32 / SZ));
}
template <int SZ>
__host__ __device__ constexpr double sin_2pi(int t) { return cos_2pi<SZ>(t - SZ / 4); }

// The lane patch of a support size.
template <int SZ> struct Shape;
template <> struct Shape<8> { static constexpr int RP = 1, CP = 2; };
template <> struct Shape<16> { static constexpr int RP = 1, CP = 8; };
template <> struct Shape<24> { static constexpr int RP = 6, CP = 3; };

template <int SZ>
constexpr bool is_pow2() { return (SZ & (SZ - 1)) == 0; }

template <typename T, int SZ>
struct Layout {
    using T2 = typename Vec2<T>::type;
    static constexpr int SS = SZ * SZ;
    static constexpr int RP = Shape<SZ>::RP, CP = Shape<SZ>::CP, P = RP * CP;
    static_assert(P * 32 == SS, "the lane patches must tile the spectrum");
    static_assert((SZ / CP) * (SZ / RP) == 32, "one patch per lane");
    // Row strides with padding against bank conflicts: the lanes of a
    // half-warp touch several rows at once.
    static constexpr int XS = SZ + 1;                      // x, w of the support (T)
    static constexpr int YS = SZ == 24 ? 28 : SZ + 1;      // first-pass outputs (T2)
    static constexpr int WROW = SZ == 24 ? 28 : 2 * SZ + 1;   // W row: its S entries, the first CP again, pad
    static_assert(WROW >= SZ + CP - 1, "a shifted patch row is read without wrapping");
    // W rows stored twice (rows S .. 2S-1 repeat 0 .. S-1) where RP > 1, so
    // the RP rows of a shifted patch are read without a row wrap.
    static constexpr int WROWS = RP > 1 ? 2 * SZ : SZ;
    static constexpr int TTS = SZ + 1;                     // row stride of the twiddle products
    // CTA tables: w0, w_f (SS T each), e^{-j 2 pi t / S} (S T2) and, when S is
    // not a power of two, the products e^{-j 2 pi (a b mod S) / S} (S x TTS T2).
    static constexpr size_t w0_off = 0;
    static constexpr size_t wf_off = w0_off + sizeof(T) * SS;
    static constexpr size_t tw_off = wf_off + sizeof(T) * SS;
    static constexpr size_t tt_off = tw_off + sizeof(T2) * SZ;
    static constexpr size_t tt_bytes = is_pow2<SZ>() ? 0 : sizeof(T2) * SZ * TTS;
    static constexpr size_t warp0_off = (tt_off + tt_bytes + 127) & ~(size_t)127;
    // Per warp, S = 8, 16: region A = x and w of the support (prologue), then
    // the W rows; region B = the first-pass outputs Yx, Yw.  S = 24 (IN_PLACE):
    // one region that holds x and w, then (both passes accumulate in
    // registers) Yx and Yw, then the W rows.
    static constexpr size_t xw_bytes = 2 * sizeof(T) * SZ * XS;
    static constexpr size_t w_bytes = sizeof(T2) * WROWS * WROW;
    static constexpr size_t y_bytes = 2 * sizeof(T2) * SZ * YS;
    static constexpr bool IN_PLACE = SZ == 24;
    static constexpr size_t a_bytes = w_bytes > xw_bytes ? w_bytes : xw_bytes;
    static constexpr size_t region = IN_PLACE ? (a_bytes > y_bytes ? a_bytes : y_bytes) : a_bytes + y_bytes;
    // RP > 1: P entries where the lane holding the block maximum publishes its values
    static constexpr size_t pub_off = (region + 15) & ~(size_t)15;
    static constexpr size_t pub_bytes = RP > 1 ? sizeof(T2) * P : 0;
    static constexpr size_t per_warp = (pub_off + pub_bytes + 127) & ~(size_t)127;
    static constexpr size_t bytes(int warps) { return warp0_off + per_warp * (size_t)warps; }
};

// Warps per CTA: 8; FP64 at S = 24 takes 4 (shared memory per warp).  FP32
// at S = 24 runs one CTA of 20 warps per SM (at most 96 registers; 220 KB of
// shared memory): 1080p, K = 100, B = 4: 4.52 ms with 2 CTAs x 8 warps (at
// most 128 registers), 4.31 ms with 18 warps, 4.20 ms with 20.
template <typename T, int SZ>
constexpr int warps() { return (sizeof(T) == 8 && SZ == 24) ? 4 : (SZ == 24 ? 20 : 8); }

template <typename T, int SZ>
__device__ __forceinline__ void tables(const MethodArgs& mth, T* sw0, T* swf, typename Vec2<T>::type* stw,
                                       typename Vec2<T>::type* stt) {
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
        if constexpr (!is_pow2<SZ>()) {
            const int t = (m * n) % SZ;
            typename Vec2<T>::type v;
            v.x = T(cos_2pi<SZ>(t));
            v.y = T(-sin_2pi<SZ>(t));
            stt[m * Layout<T, SZ>::TTS + n] = v;
        }
    }
    for (int t = threadIdx.x; t < SZ; t += blockDim.x) {
        typename Vec2<T>::type v;
        v.x = T(cos_2pi<SZ>(t));
        v.y = T(-sin_2pi<SZ>(t));   // e^{-j 2 pi t / S}
        stw[t] = v;
    }
}

// e^{-j 2 pi (a b mod S) / S}
template <int SZ, typename T2>
__device__ __forceinline__ T2 twiddle(const T2* stw, const T2* stt, int a, int b) {
    if constexpr (is_pow2<SZ>()) return stw[(a * b) & (SZ - 1)];
    else return stt[a * (SZ + 1) + b];
}

// (i mod S) for i in (-S, S)
template <int SZ>
__device__ __forceinline__ int wrap(int i) {
    if constexpr (is_pow2<SZ>()) return i & (SZ - 1);
    else return i < 0 ? i + SZ : i;
}

// In-register radix-2 FFT of length N (a power of two <= 32), natural order
// in and out, X[k] = sum_m x[m] e^{-j 2 pi k m / N}.
template <int N, typename T>
__device__ __forceinline__ void fft_pow2(T (&re)[N], T (&im)[N]) {
    constexpr int LOG = N == 2 ? 1 : N == 4 ? 2 : N == 8 ? 3 : N == 16 ? 4 : 5;
    T ar[N], ai[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        int r = 0;
#pragma unroll
        for (int b = 0; b < LOG; ++b) r |= ((i >> b) & 1) << (LOG - 1 - b);
        ar[i] = re[r];
        ai[i] = im[r];
    }
#pragma unroll
    for (int half = 1; half < N; half *= 2) {
#pragma unroll
        for (int j = 0; j < N; j += 2 * half) {
#pragma unroll
            for (int t = 0; t < half; ++t) {
                const int tw = t * (32 / (2 * half));   // e^{-j 2 pi tw / 32}
                const T br = ar[j + t + half], bi = ai[j + t + half];
                T xr, xi;
                if (tw == 0) {
                    xr = br; xi = bi;
                } else if (tw == 8) {   // times -j
                    xr = bi; xi = -br;
                } else {
                    const T c = T(cos_2pi32(tw)), sn = T(-sin_2pi32(tw));
                    xr = br * c - bi * sn;
                    xi = br * sn + bi * c;
                }
                ar[j + t + half] = ar[j + t] - xr;
                ai[j + t + half] = ai[j + t] - xi;
                ar[j + t] = ar[j + t] + xr;
                ai[j + t] = ai[j + t] + xi;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        re[i] = ar[i];
        im[i] = ai[i];
    }
}

// In-register 24-point FFT, X[k] = sum_n x[n] e^{-j 2 pi k n / 24}, as
// 3 x 8 (n = 3 n1 + n2, k = k1 + 8 k2): three 8-point FFTs over n1, the
// twiddles e^{-j 2 pi n2 k1 / 24}, eight 3-point DFTs over n2.
template <typename T>
__device__ __forceinline__ void fft24(T (&re)[24], T (&im)[24]) {
    T yr[3][8], yi[3][8];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2) {
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
            yr[n2][n1] = re[3 * n1 + n2];
            yi[n2][n1] = im[3 * n1 + n2];
        }
        fft_pow2<8>(yr[n2], yi[n2]);
    }
    const T h = T(0.866025403784438646763723170752936183);   // sin(pi / 3)
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        // y1, y2 of this k1 times e^{-j 2 pi n2 k1 / 24}
        T br = yr[1][k1], bi = yi[1][k1], cr = yr[2][k1], ci = yi[2][k1];
        if (k1 != 0) {
            const T c1 = T(cos_2pi24(k1)), s1 = T(-cos_2pi24(k1 - 6));
            const T c2 = T(cos_2pi24(2 * k1)), s2 = T(-cos_2pi24(2 * k1 - 6));
            const T tbr = br * c1 - bi * s1, tbi = br * s1 + bi * c1;
            const T tcr = cr * c2 - ci * s2, tci = cr * s2 + ci * c2;
            br = tbr; bi = tbi; cr = tcr; ci = tci;
        }
        const T ar = yr[0][k1], ai = yi[0][k1];
        const T sr = br + cr, si = bi + ci, dr = br - cr, di = bi - ci;
        const T tr = ar - T(0.5) * sr, ti = ai - T(0.5) * si;
        re[k1] = ar + sr;
        im[k1] = ai + si;
        re[k1 + 8] = tr + h * di;    // a + w b + w^2 c, w = e^{-j 2 pi / 3}
        im[k1 + 8] = ti - h * dr;
        re[k1 + 16] = tr - h * di;
        im[k1 + 16] = ti + h * dr;
    }
}

// One block: a1-a9 for support size SZ, target B x B.
template <typename T, int SZ, int B>
__device__ __forceinline__ void block(const ImageArgs& im, long long blk, int L, T gamma, const T* sw0,
                                      const T* swf, const typename Vec2<T>::type* stw,
                                      const typename Vec2<T>::type* stt, unsigned char* area,
                                      unsigned long long* empty, int lane) {
    using T2 = typename Vec2<T>::type;
    using Lay = Layout<T, SZ>;
    constexpr int P = Lay::P, RP = Lay::RP, CP = Lay::CP, WROW = Lay::WROW, XS = Lay::XS, YS = Lay::YS;
    constexpr int PT = TargetPix<B>::P;
    T* xs = reinterpret_cast<T*>(area);                 // prologue
    T* ws = xs + SZ * XS;
    T2* Yx = reinterpret_cast<T2*>(Lay::IN_PLACE ? area : area + Lay::a_bytes);
    T2* Yw = Yx + SZ * YS;
    T2* Wr = reinterpret_cast<T2*>(area);               // after the second pass
    T2* pub = reinterpret_cast<T2*>(area + Lay::pub_off);

    const int by = (int)(blk / im.nbx);
    const int bx = (int)(blk - (long long)by * im.nbx);
    const int y0 = by * B - L, x0 = bx * B - L;
    // this lane's patch: rows k0 .. k0+RP-1, columns l0 .. l0+CP-1
    const int k0 = (lane / (SZ / CP)) * RP, l0 = (lane % (SZ / CP)) * CP;
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
        constexpr bool FFT24 = SZ == 24 && sizeof(T) == 4;
        unsigned dmax = 0;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int i = lane + 32 * j;
            const int x = (i / SZ) * XS + i % SZ;
            const bool kn = ws[x] > T(0);
            const T d = xs[x] - mu;
            xs[x] = kn ? d * ws[x] : T(0);
            const unsigned ab = __float_as_uint((float)d) & 0x7fffffffu;
            dmax = (kn && ab > dmax) ? ab : dmax;
        }
        __syncwarp();
        T zr[P], zi[P], w0r = T(0);

        if constexpr (FFT24) {
            // ---- a3 as in the S = 32 kernel: one complex 2-D FFT of
            //      z = x + j alpha w (alpha = 2^e >= max |f - mu|), rows then
            //      columns, by lanes 0..23; Q and W separated with the
            //      conjugate-symmetry identities (exactly Hermitian) ----
            dmax = __reduce_max_sync(FULL, dmax);
            unsigned aexp = (dmax >> 23) + 1u;
            aexp = (dmax >= 0x00800000u && dmax < 0x7e000000u) ? aexp : 127u;
            const T alpha = T(__uint_as_float(aexp << 23));
            const T inv2alpha = T(__uint_as_float((253u - aexp) << 23));   // 1 / (2 alpha)
            constexpr int FS = 25;   // row stride (T2) of the first-pass output: conflict-free rows and columns
            T2* Yz = reinterpret_cast<T2*>(area) + SZ * WROW;   // in the second copy of the W rows
            const int rl = lane < SZ ? lane : SZ - 1;            // lanes 24..31 repeat row / column 23
            T fr[SZ], fi[SZ];
#pragma unroll
            for (int n = 0; n < SZ; ++n) {
                fr[n] = xs[rl * XS + n];
                fi[n] = ws[rl * XS + n] * alpha;
            }
            fft24(fr, fi);   // lane m: Y[m][l] = sum_n z[m][n] e^{-j 2 pi l n / 24}
            if (lane < SZ) {
#pragma unroll
                for (int l = 0; l < SZ; ++l) Yz[lane * FS + l] = make_float2(fr[l], fi[l]);
            }
            __syncwarp();
#pragma unroll
            for (int m = 0; m < SZ; ++m) {
                const T2 y = Yz[m * FS + rl];
                fr[m] = y.x;
                fi[m] = y.y;
            }
            fft24(fr, fi);   // lane l: Z[k][l], k = 0..23
            __syncwarp();    // the first-pass output is read no more
            // Q[k][l] = (Z[k][l] + conj Z[-k][-l]) / 2, W[k][l] = (Z[k][l] - conj Z[-k][-l]) / (2j alpha);
            // Z[-k][-l] is register -k of the lane holding column -l
            const int src = (SZ - rl) % SZ;
            T2* Qt = Yz;   // Q goes through the same place to the lanes' patches
#pragma unroll
            for (int k = 0; k <= SZ / 2; ++k) {
                const int k2 = (SZ - k) % SZ;
                const T cr = __shfl_sync(FULL, fr[k2], src);
                const T ci = __shfl_sync(FULL, fi[k2], src);
                T dr = cr, di = ci;
                if (k2 != k) {
                    dr = __shfl_sync(FULL, fr[k], src);
                    di = __shfl_sync(FULL, fi[k], src);
                }
                if (lane < SZ) {
                    const T ar = fr[k], ai = fi[k];
                    const T2 w1 = make_float2((ai + ci) * inv2alpha, (cr - ar) * inv2alpha);
                    Wr[k * WROW + lane] = w1;
                    if (lane < CP) Wr[k * WROW + SZ + lane] = w1;
                    Qt[k * FS + lane] = make_float2((ar + cr) * T(0.5), (ai - ci) * T(0.5));
                    if (k == 0 && lane == 0) w0r = w1.x;
                    if (k2 != k) {
                        const T br = fr[k2], bi = fi[k2];
                        const T2 w2 = make_float2((bi + di) * inv2alpha, (dr - br) * inv2alpha);
                        Wr[k2 * WROW + lane] = w2;
                        if (lane < CP) Wr[k2 * WROW + SZ + lane] = w2;
                        Qt[k2 * FS + lane] = make_float2((br + dr) * T(0.5), (bi - di) * T(0.5));
                    }
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < RP; ++r)
#pragma unroll
                for (int j = 0; j < CP; ++j) {
                    const T2 q = Qt[(k0 + r) * FS + l0 + j];
                    zr[r * CP + j] = q.x;
                    zi[r * CP + j] = q.y;
                }
            __syncwarp();
            // the second copy of the W rows (rows S .. 2S-1 repeat 0 .. S-1)
            for (int e = lane; e < SZ * WROW; e += 32) Wr[SZ * WROW + e] = Wr[e];
        } else {
        // ---- a3, pass 1 (over n): Y[m][l] = sum_n v[m][n] e^{-j 2 pi l n / S},
        //      for the rows m and columns l of this lane's patch ----
        if constexpr (RP == 1) {
            T xr[SZ], wr_[SZ];
#pragma unroll
            for (int n = 0; n < SZ; ++n) {
                xr[n] = xs[k0 * XS + n];
                wr_[n] = ws[k0 * XS + n];
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const int l = l0 + p;
                T axr = T(0), axi = T(0), awr = T(0), awi = T(0);
#pragma unroll
                for (int n = 0; n < SZ; ++n) {
                    const T2 t = twiddle<SZ>(stw, stt, l, n);
                    axr = fma_rn(xr[n], t.x, axr);
                    axi = fma_rn(xr[n], t.y, axi);
                    awr = fma_rn(wr_[n], t.x, awr);
                    awi = fma_rn(wr_[n], t.y, awi);
                }
                T2 vx, vw;
                vx.x = axr; vx.y = axi;
                vw.x = awr; vw.y = awi;
                Yx[k0 * YS + l] = vx;
                Yw[k0 * YS + l] = vw;
            }
        } else {
            T axr[P], axi[P], awr[P], awi[P];
#pragma unroll
            for (int p = 0; p < P; ++p) axr[p] = axi[p] = awr[p] = awi[p] = T(0);
#pragma unroll 1
            for (int n = 0; n < SZ; ++n) {
                T2 t[CP];
#pragma unroll
                for (int j = 0; j < CP; ++j) t[j] = twiddle<SZ>(stw, stt, l0 + j, n);
#pragma unroll
                for (int r = 0; r < RP; ++r) {
                    const T xv = xs[(k0 + r) * XS + n], wv = ws[(k0 + r) * XS + n];
#pragma unroll
                    for (int j = 0; j < CP; ++j) {
                        const int p = r * CP + j;
                        axr[p] = fma_rn(xv, t[j].x, axr[p]);
                        axi[p] = fma_rn(xv, t[j].y, axi[p]);
                        awr[p] = fma_rn(wv, t[j].x, awr[p]);
                        awi[p] = fma_rn(wv, t[j].y, awi[p]);
                    }
                }
            }
            if constexpr (Lay::IN_PLACE) __syncwarp();   // x, w are read no more: Y goes there
#pragma unroll
            for (int r = 0; r < RP; ++r)
#pragma unroll
                for (int j = 0; j < CP; ++j) {
                    const int p = r * CP + j;
                    T2 vx, vw;
                    vx.x = axr[p]; vx.y = axi[p];
                    vw.x = awr[p]; vw.y = awi[p];
                    Yx[(k0 + r) * YS + l0 + j] = vx;
                    Yw[(k0 + r) * YS + l0 + j] = vw;
                }
        }
        __syncwarp();

        // ---- a3, pass 2 (over m): Z[k][l] = sum_m Y[m][l] e^{-j 2 pi k m / S} ----
        {
            T2 wv[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                zr[p] = zi[p] = T(0);
                wv[p].x = wv[p].y = T(0);
            }
#pragma unroll
            for (int m = 0; m < SZ; ++m) {
                T2 t[RP];
#pragma unroll
                for (int r = 0; r < RP; ++r) t[r] = twiddle<SZ>(stw, stt, k0 + r, m);
#pragma unroll
                for (int j = 0; j < CP; ++j) {
                    const T2 a = Yx[m * YS + l0 + j];
                    const T2 b = Yw[m * YS + l0 + j];
#pragma unroll
                    for (int r = 0; r < RP; ++r) {
                        const int p = r * CP + j;
                        zr[p] = fma_rn(a.x, t[r].x, fma_rn(-a.y, t[r].y, zr[p]));
                        zi[p] = fma_rn(a.x, t[r].y, fma_rn(a.y, t[r].x, zi[p]));
                        wv[p].x = fma_rn(b.x, t[r].x, fma_rn(-b.y, t[r].y, wv[p].x));
                        wv[p].y = fma_rn(b.x, t[r].y, fma_rn(b.y, t[r].x, wv[p].y));
                    }
                }
            }
            __syncwarp();   // the region the W rows go to is read no more
#pragma unroll
            for (int r = 0; r < RP; ++r)
#pragma unroll
                for (int j = 0; j < CP; ++j) {
                    const int p = r * CP + j;
                    Wr[(k0 + r) * WROW + l0 + j] = wv[p];
                    if (l0 + j < CP) Wr[(k0 + r) * WROW + SZ + l0 + j] = wv[p];
                    if constexpr (Lay::WROWS > SZ) {
                        Wr[(SZ + k0 + r) * WROW + l0 + j] = wv[p];
                        if (l0 + j < CP) Wr[(SZ + k0 + r) * WROW + SZ + l0 + j] = wv[p];
                    }
                }
            if (lane == 0) w0r = wv[0].x;   // W[0][0] (component 0 of lane 0)
        }
        }   // direct DFTs
        const T W0 = __shfl_sync(FULL, w0r, 0);
        __syncwarp();

        // ---- a4-a8 ----
        T wfv[P];
#pragma unroll
        for (int r = 0; r < RP; ++r)
#pragma unroll
            for (int j = 0; j < CP; ++j) wfv[r * CP + j] = swf[(k0 + r) * SZ + l0 + j];
        // the published entry lane t < P examines, and its w_f offset within the patch
        const int lane_pub = lane < P ? lane : P - 1;
        const int lane_wf = (lane_pub / CP) * SZ + lane_pub % CP;
        int pm[PT], pn[PT];
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            pm[q] = L + (lane + 32 * q) / B;
            pn[q] = L + (lane + 32 * q) % B;
        }
        const T invW0 = T(1) / W0;
        const T cg = gamma * invW0;   // FP32: c = R[u,v] gamma / W[0,0] (Eqs. 10, 11)
        // o[] is written by every pass before block_max reads it; the front
        // end cannot see that through the lambdas (diagnostic 549)
#pragma nv_diag_suppress 549
        T o[P];
        int nu = 0;
        T cr = T(0), ci = T(0);
        int u = 0, v = 0;
        T ar = mu, ai = T(0);   // DC phase: R = a W + Q

        T sr, si;   // the picked component's value

        // a5 for the objectives o[] of this lane's components with values
        // (vr, vi): block maximum, then the lowest linear index holding it;
        // sets u, v and (sr, si).
        T mx, Mx;
        // block maximum of the objectives o[]: this lane's (mx) and the warp's (Mx)
        auto block_max = [&]() {
            if constexpr (sizeof(T) == 4 && P == 8) {
                mx = max3(max3(o[0], o[1], o[2]), max3(o[3], o[4], o[5]), fmaxf(o[6], o[7]));
            } else if constexpr (sizeof(T) == 4) {
                mx = o[0];
#pragma unroll
                for (int p = 1; p + 1 < P; p += 2) mx = max3(mx, o[p], o[p + 1]);
                if constexpr ((P - 1) % 2 != 0) mx = fmaxf(mx, o[P - 1]);
            } else {
                mx = o[0];
#pragma unroll
                for (int p = 1; p < P; ++p) mx = fmax(mx, o[p]);
            }
            Mx = mx;
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
        };
        // a5 after block_max: the lowest linear index holding Mx among this
        // lane's components with values (vr, vi); sets u, v and (sr, si).
        auto pick = [&](const T (&vr)[P], const T (&vi)[P]) {
            int c;
            sr = vr[P - 1];
            si = vi[P - 1];
            if constexpr (RP == 1) {
                // lanes and registers are in linear order: lowest lane, then lowest register
                const int ul = __ffs(__ballot_sync(FULL, mx == Mx)) - 1;
                int pf = P - 1;
#pragma unroll
                for (int p = P - 2; p >= 0; --p) {
                    const bool hit = o[p] == Mx;
                    pf = hit ? p : pf;
                    sr = hit ? vr[p] : sr;
                    si = hit ? vi[p] : si;
                }
                pf = __shfl_sync(FULL, pf, ul);
                sr = __shfl_sync(FULL, sr, ul);
                si = __shfl_sync(FULL, si, ul);
                c = ul * P + pf;
            } else {
                // registers are in row-major order within the patch: the lane's
                // first hit is its lowest linear index; the warp minimum of the
                // lanes' candidates is the block's
                unsigned cand = 0x7fff0000u;
#pragma unroll
                for (int p = P - 1; p >= 0; --p) {
                    const bool hit = o[p] == Mx;
                    cand = hit ? (unsigned)((p / CP) * SZ + p % CP) : cand;
                    sr = hit ? vr[p] : sr;
                    si = hit ? vi[p] : si;
                }
                cand += (unsigned)(k0 * SZ + l0);
                unsigned cmin = __reduce_min_sync(FULL, cand);
                const int ul = __ffs(__ballot_sync(FULL, cand == cmin)) - 1;
                if (cmin >= (unsigned)(SZ * SZ)) cmin = 0;   // no lane matched (NaN objective): stay in range
                sr = __shfl_sync(FULL, sr, ul);
                si = __shfl_sync(FULL, si, ul);
                c = (int)cmin;
            }
            u = c / SZ;
            v = c % SZ;
        };
        auto select = [&](const T (&vr)[P], const T (&vi)[P]) {
            block_max();
            pick(vr, vi);
        };
        // a6 for the picked component: c, the recorded index, the target pixels.
        auto apply = [&]() {
            if constexpr (sizeof(T) == 4) {
                cr = sr * cg;
                ci = si * cg;
            } else {   // FP64 debug: gamma (R / W[0,0]) in the oracle's order
                cr = gamma * (sr * invW0);
                ci = gamma * (si * invW0);
            }
            if (seq != nullptr && lane == 0) seq[nu] = (int16_t)(u * SZ + v);
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                int ph;
                if constexpr (is_pow2<SZ>()) ph = (SZ - ((u * pm[q] + v * pn[q]) & (SZ - 1))) & (SZ - 1);
                else {
                    ph = (u * pm[q] + v * pn[q]) % SZ;
                    ph = ph == 0 ? 0 : SZ - ph;
                }
                const T2 e = stw[ph];   // e^{+j 2 pi (u m + v n) / S}
                gacc[q] = fma_rn(cr, e.x, fma_rn(-ci, e.y, gacc[q]));   // Re(c e^{+j theta})
            }
        };

        // ---- DC phase: R = a W + Q ----
        bool done = im.K <= 0;
        if (!done) {
            for (;;) {
                if constexpr (RP == 1) {
                    T rr[P], ri[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const T2 w = Wr[k0 * WROW + l0 + p];
                        split_value(ar, ai, w.x, w.y, zr[p], zi[p], rr[p], ri[p]);
                        o[p] = objective<T>(rr[p], ri[p], wfv[p]);
                    }
                    select(rr, ri);
                } else {
#pragma unroll
                    for (int r = 0; r < RP; ++r)
#pragma unroll
                        for (int j = 0; j < CP; ++j) {
                            const int p = r * CP + j;
                            const T2 w = Wr[(k0 + r) * WROW + l0 + j];
                            T rr_, ri_;
                            split_value(ar, ai, w.x, w.y, zr[p], zi[p], rr_, ri_);
                            o[p] = objective<T>(rr_, ri_, wfv[p]);
                        }
                    // the scan held Q: form the picked value a W[u][v] + Q[u][v]
                    // with the same rounded operations
                    select(zr, zi);
                    const T2 w = Wr[u * WROW + v];
                    T rr_, ri_;
                    split_value(ar, ai, w.x, w.y, sr, si, rr_, ri_);
                    sr = rr_;
                    si = ri_;
                }
                apply();
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
                for (int r = 0; r < RP; ++r)
#pragma unroll
                    for (int j = 0; j < CP; ++j) {
                        const int p = r * CP + j;
                        const T2 w = Wr[(k0 + r) * WROW + l0 + j];
                        split_value(ar, ai, w.x, w.y, zr[p], zi[p], zr[p], zi[p]);
                    }
            }
        }
        // ---- a7 (Eq. 12) for the last pick and the next objective, a5-a6 ----
        while (!done) {
            const int lc = wrap<SZ>(l0 - v);
            // rows k0 - u + r (mod S): one base for the doubled rows
            const T2* base = Wr + (RP > 1 ? k0 - u + SZ : 0) * WROW + lc;
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                const T2* row = RP > 1 ? base + r * WROW : Wr + wrap<SZ>(k0 + r - u) * WROW + lc;
#pragma unroll
                for (int j = 0; j < CP; ++j) {
                    const int p = r * CP + j;
                    const T2 w = row[j];
                    residual_update(zr[p], zi[p], w.x, w.y, cr, ci);
                    o[p] = objective<T>(zr[p], zi[p], wfv[p]);
                }
            }
            if constexpr (RP == 1) {
                select(zr, zi);
            } else {
                block_max();
                const unsigned cands = __ballot_sync(FULL, mx == Mx);
                if (__popc(cands) == 1) {
                    // One lane holds the block maximum: it publishes its values,
                    // and lane t < P forms the objective of that lane's component
                    // t again (the same rounded operations and w_f entry), so the
                    // first lane that meets Mx has the lowest linear index.
                    const int ul = __ffs(cands) - 1;
                    __syncwarp();   // the previous pick's reads of pub are done
                    if (lane == ul) {
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            T2 e;
                            e.x = zr[p];
                            e.y = zi[p];
                            pub[p] = e;
                        }
                    }
                    __syncwarp();
                    const int kw = (ul / (SZ / CP)) * RP, lw = (ul % (SZ / CP)) * CP;
                    const T2 rv = pub[lane_pub];
                    const bool hit = lane < P && objective<T>(rv.x, rv.y, swf[kw * SZ + lw + lane_wf]) == Mx;
                    int pf = __ffs(__ballot_sync(FULL, hit)) - 1;
                    if (pf < 0) pf = 0;   // unreachable: the lane's maximum is one of its objectives
                    sr = __shfl_sync(FULL, rv.x, pf);
                    si = __shfl_sync(FULL, rv.y, pf);
                    u = kw + pf / CP;
                    v = lw + pf % CP;
                } else {
                    pick(zr, zi);   // ties across lanes, or no lane matched
                }
            }
            apply();
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

template <typename T, int SZ, int B>
__device__ __forceinline__ void run(const BatchArgs& a) {
    using Lay = Layout<T, SZ>;
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    T* sw0 = reinterpret_cast<T*>(smem + Lay::w0_off);
    T* swf = reinterpret_cast<T*>(smem + Lay::wf_off);
    T2* stw = reinterpret_cast<T2*>(smem + Lay::tw_off);
    T2* stt = reinterpret_cast<T2*>(smem + Lay::tt_off);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char* area = smem + Lay::warp0_off + Lay::per_warp * warp;
    tables<T, SZ>(a.mth, sw0, swf, stw, stt);
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
            block<T, SZ, B>(im, item - __ldg(a.first + lo), a.mth.L, gamma, sw0, swf, stw, stt, area, a.empty,
                            lane);
        }
    }
}

// One CTA per SM by launch bounds (the register count is the compiler's,
// at most 65536 / (32 WARPS)).
template <typename T, int SZ, int B, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) fsr_small_kernel(const BatchArgs a) {
    run<T, SZ, B>(a);
}

template <typename T, int SZ, int B>
constexpr auto kernel_of() {
    return fsr_small_kernel<T, SZ, B, warps<T, SZ>()>;
}

template <typename T, int SZ, int B>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(kernel_of<T, SZ, B>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Layout<T, SZ>::bytes(warps<T, SZ>()));
}

template <typename T, int SZ, int B>
cudaError_t launch_one(const BatchArgs& a, int chunk, int sm_count, cudaStream_t stream) {
    constexpr int W = warps<T, SZ>();
    const size_t smem = Layout<T, SZ>::bytes(W);
    auto k = kernel_of<T, SZ, B>();
    int grid = 0;
    cudaError_t e = persistent_grid(k, W, smem, (a.total + chunk - 1) / chunk, sm_count, &grid);
    if (e != cudaSuccess) return e;
    k<<<grid, W * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace small
}  // namespace fsrk
