// FP32 FSR with a support S in {4, 8, 16} (B <= S; the support-size study of
// Sec. IV, Figs. 3 and 5): one group of S lanes per block, 32 / S blocks per
// warp.  Lane t of a group holds column t of the support, then row t of the
// spectrum (S complex values in registers), as the S = 32 kernel does with a
// whole warp:
//   a1-a3  the support is loaded by columns, the weighted mean mu is removed,
//          x = (f - mu) w and alpha w are packed into z = x + j alpha w, and
//          the 2-D DFT of Eq. (7) is two in-register radix-2 FFTs of length
//          S with a transpose through shared memory; R_w and W are formed
//          from Z[k][l] and conj Z[-k][-l] with commutative operations, so
//          both are exactly Hermitian (the ties of the first iteration are
//          exact, as in the oracle);
//   a4-a8  R = a W + Q while only the DC component is selected (DC phase),
//          then Q alone; Eq. (12) reads the shifted W row of 2S - 1 stored
//          entries (the first S - 1 repeated: no column wrap) with 8-byte
//          loads; the rows (2S + 1 entries) and the per-block regions (sized
//          = S mod 16 entries) keep the loads of the groups sharing a
//          half-warp on distinct bank pairs; the objective of Eq. (8) is
//          rounded explicitly; the lane holding the block maximum publishes
//          its row in shared memory and lane t of the group forms the
//          objective of component t again, so the lowest index with the
//          maximum is found by two ballots;
//   a9     Re g (sparse inverse of G) accumulated at the target pixels only.
// The blocks of a warp may have different K and leave the DC phase at
// different iterations: the loop runs to the largest K and every step that is
// specific to one group is plain arithmetic on its lanes; every shuffle,
// ballot and warp barrier is reached by all 32 lanes.
#include "fsr_launch.h"

namespace fsrk {
namespace {

template <int SZ>
struct Grp {
    static_assert(SZ == 4 || SZ == 8 || SZ == 16, "group kernels cover S = 4, 8, 16");
    static constexpr int WS = 2 * SZ + 1;            // W row stride (float2)
    static constexpr int TS = SZ + 1;                // transpose stride (float2)
    static constexpr int WFS = SZ + 1;               // w_f row stride (float)
    static constexpr int BPW = 32 / SZ;              // blocks per warp
    static constexpr unsigned LOW = (SZ == 32) ? 0xFFFFFFFFu : ((1u << SZ) - 1u);
    static constexpr int WAREA = SZ * WS;            // float2: W rows, also the transpose
    static_assert(SZ * TS <= WAREA, "the transpose fits in the W area");
    static_assert(WAREA % 2 == 0, "the published row is 16-byte aligned");
    // per-block region (float2): W area + published row, padded to = S mod 16
    static constexpr int REGION0 = WAREA + SZ;
    static constexpr int REGION = SZ >= 16 ? REGION0 : REGION0 + ((SZ - REGION0 % 16) + 16) % 16;
    static_assert(SZ >= 16 || REGION % 16 == SZ, "regions of the groups of a half-warp on distinct bank pairs");
    static constexpr size_t w0_off = 0;
    static constexpr size_t wf_off = w0_off + 4 * SZ * SZ;
    // w_f again with one copy per group of a warp side by side in 32-word
    // rows: group g reads its copy at words 32 u + S g + t, on banks no other
    // group of the warp touches, whatever row u it picked (1080p: S = 8
    // 0.702 -> 0.683 ms, S = 16 1.797 -> 1.776 ms)
    static constexpr size_t wfg_off = wf_off + 4 * SZ * WFS;
    static constexpr size_t cs_off = wfg_off + 4 * SZ * 32;
    static constexpr size_t warp0_off = (cs_off + 8 * SZ + 127) & ~(size_t)127;
    static constexpr size_t per_warp = (size_t)8 * REGION * BPW;
    static constexpr size_t bytes(int warps) { return warp0_off + per_warp * (size_t)warps; }
};

template <int N>
__host__ __device__ constexpr int bit_reverse(int i) {
    int r = 0;
    for (int b = 1, rb = N >> 1; b < N; b <<= 1, rb >>= 1)
        if (i & b) r |= rb;
    return r;
}

// In-register radix-2 decimation-in-time FFT of length N, natural order in
// and out, X[k] = sum_m x[m] e^{-j 2 pi k m / N}.
template <int N>
__device__ __forceinline__ void fftn(float (&re)[N], float (&im)[N]) {
    float ar[N], ai[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        ar[i] = re[bit_reverse<N>(i)];
        ai[i] = im[bit_reverse<N>(i)];
    }
#pragma unroll
    for (int half = 1; half < N; half *= 2) {
#pragma unroll
        for (int j = 0; j < N; j += 2 * half) {
#pragma unroll
            for (int t = 0; t < half; ++t) {
                const int tw = t * (N / 2 / half);   // e^{-j 2 pi tw / N}
                const float br = ar[j + t + half], bi = ai[j + t + half];
                float xr, xi;
                if (tw == 0) {
                    xr = br;
                    xi = bi;
                } else if (tw == N / 4) {   // times -j
                    xr = bi;
                    xi = -br;
                } else {
                    const float c = float(cos_2pi32(tw * (32 / N))), s = float(-sin_2pi32(tw * (32 / N)));
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
    for (int i = 0; i < N; ++i) {
        re[i] = ar[i];
        im[i] = ai[i];
    }
}

// butterfly reductions inside a group of SZ lanes
template <int SZ>
__device__ __forceinline__ unsigned group_umax(unsigned v) {
#pragma unroll
    for (int s = SZ / 2; s > 0; s >>= 1) v = max(v, (unsigned)__shfl_xor_sync(FULL, v, s));
    return v;
}
template <int SZ>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int s = SZ / 2; s > 0; s >>= 1) v += __shfl_xor_sync(FULL, v, s);
    return v;
}

template <int SZ>
__device__ __forceinline__ float wf_row(const float (&wfr)[SZ / 2 + 1], int l) {
    return wfr[l <= SZ / 2 ? l : SZ - l];
}

template <int N>
__device__ __forceinline__ float max_all(const float (&o)[N]) {
    float m = fmaxf(o[0], o[1]);
#pragma unroll
    for (int l = 2; l < N; l += 2) m = max3(m, o[l], o[l + 1]);
    return m;
}

// maximum of the objective over the lane's row of R = a W + Q (unshifted W row)
template <int SZ>
__device__ __forceinline__ float split_objective_row(const float (&zr)[SZ], const float (&zi)[SZ],
                                                     const float (&wfr)[SZ / 2 + 1], const float2* wrow, float ar,
                                                     float ai) {
    float o[SZ];
#pragma unroll
    for (int l = 0; l < SZ; ++l) {
        const float2 w = wrow[l];
        float rr, ri;
        split_value(ar, ai, w.x, w.y, zr[l], zi[l], rr, ri);
        o[l] = objective<float>(rr, ri, wf_row<SZ>(wfr, l));
    }
    return max_all(o);
}

template <int SZ, int B>
__device__ __forceinline__ void group_block(const ImageArgs& im, long long blk, bool valid, int Kmax, int L,
                                            float gamma, const float* __restrict__ sw0,
                                            const float* __restrict__ swf, const float* __restrict__ swfg,
                                            const float2* __restrict__ scs,
                                            float2* Wd, float2* rowbuf, unsigned long long* empty, int lane) {
    using G = Grp<SZ>;
    constexpr int WS = G::WS, TS = G::TS, WFS = G::WFS;
    constexpr int PT = (B * B + SZ - 1) / SZ;   // target pixels per lane
    const int t = lane & (SZ - 1), gb = lane & ~(SZ - 1);
    int by = 0, bx = 0;
    if (valid) {
        by = (int)(blk / im.nbx);
        bx = (int)(blk - (long long)by * im.nbx);
    }
    const int y0 = by * B - L, x0 = bx * B - L;

    // ---- a1, a2: column t of the support, weights, weighted mean ----
    float zr[SZ], zi[SZ];
    unsigned known = 0;
    const int x = x0 + t;
#pragma unroll
    for (int m = 0; m < SZ; ++m) {
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
    for (int m = 0; m < SZ; ++m) {
        const float w = ((known >> m) & 1u) ? sw0[m * SZ + t] : 0.f;
        sw += w;
        sfw += w * zr[m];
    }
    sw = group_sum<SZ>(sw);
    sfw = group_sum<SZ>(sfw);
    const unsigned kb = (__ballot_sync(FULL, known != 0) >> gb) & G::LOW;
    const bool active = valid && kb != 0u;
    const float mu = active ? sfw / sw : 0.f;
    unsigned dmax = 0;
#pragma unroll
    for (int m = 0; m < SZ; ++m) {
        const bool kn = (known >> m) & 1u;
        const float w = kn ? sw0[m * SZ + t] : 0.f;
        const float d = zr[m] - mu;
        zr[m] = kn ? d * w : 0.f;
        zi[m] = w;
        const unsigned ab = __float_as_uint(d) & 0x7fffffffu;
        dmax = (kn && ab > dmax) ? ab : dmax;
    }
    // alpha = 2^e >= max |f - mu|: both halves of z = x + j alpha w have one
    // magnitude through the shared FFT; powers of two are undone exactly
    dmax = group_umax<SZ>(dmax);
    unsigned aexp = (dmax >> 23) + 1u;
    aexp = (dmax >= 0x00800000u && dmax < 0x7e000000u) ? aexp : 127u;
    const float alpha = __uint_as_float(aexp << 23);
    const float inv2alpha = __uint_as_float((253u - aexp) << 23);
#pragma unroll
    for (int m = 0; m < SZ; ++m) zi[m] *= alpha;

    // ---- a3: FFT over m (lane t holds column t), transpose, FFT over n ----
    fftn<SZ>(zr, zi);
    __syncwarp();   // the W area of the previous blocks is free
#pragma unroll
    for (int k = 0; k < SZ; ++k) Wd[k * TS + t] = make_float2(zr[k], zi[k]);
    __syncwarp();
#pragma unroll
    for (int n = 0; n < SZ; ++n) {
        const float2 v = Wd[t * TS + n];
        zr[n] = v.x;
        zi[n] = v.y;
    }
    __syncwarp();
    fftn<SZ>(zr, zi);   // lane k = t holds Z[k][0..S-1]

    // Q[k][l] = (Z[k][l] + conj Z[-k][-l]) / 2,  W[k][l] = (Z[k][l] - conj Z[-k][-l]) / (2j alpha)
    const int src = gb + ((SZ - t) & (SZ - 1));
    float2* wrow_out = Wd + t * WS;
    float w00 = 0.f;
#pragma unroll
    for (int l = 0; l <= SZ / 2; ++l) {
        const int l2 = (SZ - l) & (SZ - 1);
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
        if (l < SZ - 1) wrow_out[l + SZ] = w1;
        if (l == 0) w00 = w1.x;
        if (l2 != l) {
            const float br = zr[l2], bi = zi[l2];
            const float2 w2 = make_float2((bi + di) * inv2alpha, (dr - br) * inv2alpha);
            zr[l2] = (br + dr) * 0.5f;
            zi[l2] = (bi - di) * 0.5f;
            wrow_out[l2] = w2;
            if (l2 < SZ - 1) wrow_out[l2 + SZ] = w2;
        }
    }
    const float W0 = __shfl_sync(FULL, w00, gb);
    __syncwarp();

    // ---- a4-a8 ----
    float wfr[SZ / 2 + 1];
#pragma unroll
    for (int l = 0; l <= SZ / 2; ++l) wfr[l] = swf[t * WFS + l];
    int pm[PT], pn[PT];
    float gacc[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        pm[q] = L + (t + SZ * q) / B;
        pn[q] = L + (t + SZ * q) % B;
        gacc[q] = 0.f;
    }
    const int Kh = valid ? im.K : 0;
    int16_t* seq = (valid && im.seq) ? im.seq + (size_t)blk * im.K : nullptr;
    if (valid && !active && t == 0) empty_block(seq, im.K, empty);
    const float cg = active ? gamma * (1.f / W0) : 0.f;   // c = R[u,v] gamma / W[0,0] (Eqs. 10, 11)
    bool split = true;             // R = a W + Q (DC phase)
    float ar = mu, ai = 0.f;
    float m_lane = (active && Kh > 0) ? split_objective_row<SZ>(zr, zi, wfr, Wd + t * WS, ar, ai) : 0.f;

    // One iteration; dc = false when no running group of the warp is in its
    // DC phase (the split branches then drop out at compile time).
    auto step = [&](int nu, bool dc, bool all) {
        // all: every group of the warp holds an active block with K = Kmax,
        // so the per-group run conditions drop out at compile time
        const bool run = all || (active && nu < Kh);
        const int Kr = all ? Kmax : Kh;
        // a5: block maximum (each group reduces over its own lanes), the
        // lowest row holding it, then its lowest column
        // (a butterfly over the group's lanes: a warp reduction with the
        // group's lane mask runs once per group; 1080p: S = 4 0.366 -> 0.270
        // ms, S = 8 0.718 -> 0.705 ms, S = 16 1.842 -> 1.798 ms)
        const unsigned Mb = group_umax<SZ>(run ? __float_as_uint(m_lane) : 0u);
        const unsigned ub = (__ballot_sync(FULL, run && __float_as_uint(m_lane) == Mb) >> gb) & G::LOW;
        const int u = ub ? __ffs(ub) - 1 : 0;
        __syncwarp();   // the previous pick's reads of the published row are done
        if (run && t == u) {
            float4* pub = reinterpret_cast<float4*>(rowbuf);
#pragma unroll
            for (int i = 0; i < SZ / 2; ++i) pub[i] = make_float4(zr[2 * i], zi[2 * i], zr[2 * i + 1], zi[2 * i + 1]);
        }
        __syncwarp();
        const float2 qv = rowbuf[t];
        float rr = qv.x, ri = qv.y;
        if (dc && split) {
            const float2 w = Wd[u * WS + t];
            split_value(ar, ai, w.x, w.y, qv.x, qv.y, rr, ri);
        }
        const float o = objective<float>(rr, ri, swfg[u * 32 + gb + t]);
        const unsigned vbits = (__ballot_sync(FULL, run && __float_as_uint(o) == Mb) >> gb) & G::LOW;
        const int v = vbits ? __ffs(vbits) - 1 : 0;
        const float Rr = __shfl_sync(FULL, rr, gb + v);
        const float Ri = __shfl_sync(FULL, ri, gb + v);

        // a6 (Eqs. 10, 11): c = gamma p, the target pixels of the sparse inverse
        const float cr = Rr * cg, ci = Ri * cg;
        if (run) {
            if (seq != nullptr && t == 0) seq[nu] = (int16_t)(u * SZ + v);
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const float2 cs = scs[(u * pm[q] + v * pn[q]) & (SZ - 1)];
                gacc[q] = fma_rn(cr, cs.x, fma_rn(-ci, cs.y, gacc[q]));
            }
        }
        // a7 (Eq. 12) and the objective of the next iteration (this group only)
        if (run && nu + 1 < Kr) {
            if (dc && split && (u | v) == 0) {
                ar -= cr;
                ai -= ci;
                m_lane = split_objective_row<SZ>(zr, zi, wfr, Wd + t * WS, ar, ai);
            } else {
                if (dc && split) {   // fold a W into Q
                    const float2* wk = Wd + t * WS;
#pragma unroll
                    for (int l = 0; l < SZ; ++l) {
                        const float2 w = wk[l];
                        split_value(ar, ai, w.x, w.y, zr[l], zi[l], zr[l], zi[l]);
                    }
                    split = false;
                }
                const float2* row = Wd + ((t - u) & (SZ - 1)) * WS + ((SZ - v) & (SZ - 1));
                float o2[SZ];
#pragma unroll
                for (int l = 0; l < SZ; ++l) {
                    const float2 w = row[l];
                    residual_update(zr[l], zi[l], w.x, w.y, cr, ci);
                    o2[l] = objective<float>(zr[l], zi[l], wf_row<SZ>(wfr, l));
                }
                m_lane = max_all(o2);
            }
        }
    };
    // the loops run to the largest K of the warp (uniform): a DC loop, then a
    // loop without the split branches (1080p frame: S = 4 0.385 -> 0.365 ms,
    // S = 8 0.776 -> 0.747 ms; S = 16 at 20 warps per SM 1.935 -> 1.922 ms,
    // at 16 warps and 123 registers 2.07 -> 2.15 ms), in a form without the
    // per-group run conditions when every group runs to the same K (S = 16
    // 1.902 -> 1.848 ms, S = 4 0.369 -> 0.358 ms; S = 8 unchanged, with 32
    // bytes spilled, so it keeps one form)
    int nu = 0;
    while (nu < Kmax && __any_sync(FULL, split && active && nu < Kh)) step(nu++, true, false);
    if constexpr (SZ != 8) {
        if (__all_sync(FULL, active && Kh == Kmax)) {
            for (; nu < Kmax; ++nu) step(nu, false, true);
        }
    }
    for (; nu < Kmax; ++nu) step(nu, false, false);


    // ---- a9: write-back of the B x B target ----
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int pidx = t + SZ * q;
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

// Warps per CTA and CTAs per SM the register budget is set for: 20 warps
// per SM at S = 16 (2 x 10, <= 96 registers, no spill), 32 at S = 8 (4 x 8,
// <= 64, 36 bytes spilled) and at S = 4 (4 x 8, <= 64, no spill).  Measured
// on the 1080p frame, K = 100: S = 4 0.53 ms with 16 warps per SM, 0.39 ms
// with 32; S = 8 0.91 ms with 16, 0.745 ms with 24 (3 x 8), 0.722 ms with
// 32; S = 16 2.07 ms with 16 (2 x 8), 1.93 ms with 20 (2 x 10 or 4 x 5),
// 2.19 ms with 21 (3 x 7), 2.13 ms with 24 (2 x 12, 52 bytes spilled).
template <int SZ> constexpr int group_warps() { return SZ == 16 ? 10 : 8; }
template <int SZ> constexpr int group_min_ctas() { return SZ == 16 ? 2 : 4; }

template <int SZ, int B, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, group_min_ctas<SZ>()) fsr_group_kernel(const BatchArgs a) {
    using G = Grp<SZ>;
    extern __shared__ __align__(128) unsigned char smem[];
    float* sw0 = reinterpret_cast<float*>(smem + G::w0_off);
    float* swf = reinterpret_cast<float*>(smem + G::wf_off);
    float2* scs = reinterpret_cast<float2*>(smem + G::cs_off);
    float* swfg = reinterpret_cast<float*>(smem + G::wfg_off);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = lane / SZ;
    float2* Wd = reinterpret_cast<float2*>(smem + G::warp0_off + G::per_warp * warp) + (size_t)G::REGION * grp;
    float2* rowbuf = Wd + G::WAREA;

    // tables: Eq. (5) without the known-set factor, Eq. (9), cos/sin(2 pi t / S)
    const float hs = float(SZ) / 2.f;
    for (int i = threadIdx.x; i < SZ * SZ; i += blockDim.x) {
        const int m = i / SZ, n = i % SZ;
        const float dm = float(m) - float(SZ - 1) / 2.f, dn = float(n) - float(SZ - 1) / 2.f;
        sw0[i] = powf(a.mth.rho, sqrtf(dm * dm + dn * dn));
        float wfv = 1.f;
        if (a.mth.freq_weight) {
            const float kt = hs - fabsf(float(m) - hs), lt = hs - fabsf(float(n) - hs);
            const float r = sqrtf(kt * kt / float(SZ * SZ) + lt * lt / float(SZ * SZ));
            const float b = 1.f - sqrtf(2.f) * r;
            wfv = b * b;
        }
        swf[m * G::WFS + n] = wfv;
#pragma unroll
        for (int g = 0; g < G::BPW; ++g) swfg[m * 32 + g * SZ + n] = wfv;
    }
    for (int i = threadIdx.x; i < SZ; i += blockDim.x)
        scs[i] = make_float2(float(cos_2pi32(i * (32 / SZ))), float(sin_2pi32(i * (32 / SZ))));
    __syncthreads();

    const float gamma = a.mth.gamma;
    const long long take = (long long)G::BPW * a.chunk;   // 32 / S blocks per warp and chunk step
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.counter, (unsigned long long)take);
        base = __shfl_sync(FULL, base, 0);
        if (base >= (unsigned long long)a.total) break;
        const long long end = min((long long)base + take, a.total);
        for (long long first = (long long)base; first < end; first += G::BPW) {
            const long long item = first + grp;
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
            int Kmax = valid ? im.K : 0;
#pragma unroll
            for (int s = 16; s >= SZ; s >>= 1) Kmax = max(Kmax, __shfl_xor_sync(FULL, Kmax, s));
            group_block<SZ, B>(im, blk, valid, Kmax, a.mth.L, gamma, sw0, swf, swfg, scs, Wd, rowbuf, a.empty, lane);
        }
    }
}

template <int SZ, int B>
cudaError_t configure_one() {
    constexpr int W = group_warps<SZ>();
    return cudaFuncSetAttribute(fsr_group_kernel<SZ, B, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Grp<SZ>::bytes(W));
}

template <int SZ, int B>
cudaError_t launch_one(const BatchArgs& a, int chunk, int sm_count, cudaStream_t stream) {
    constexpr int W = group_warps<SZ>();
    const size_t smem = Grp<SZ>::bytes(W);
    int grid = 0;
    const long long take = (long long)Grp<SZ>::BPW * chunk;
    cudaError_t e = persistent_grid(fsr_group_kernel<SZ, B, W>, W, smem,
                                    (a.total + take - 1) / take, sm_count, &grid);
    if (e != cudaSuccess) return e;
    fsr_group_kernel<SZ, B, W><<<grid, W * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_group() {
    cudaError_t e;
    if ((e = configure_one<16, 2>()) != cudaSuccess) return e;
    if ((e = configure_one<16, 4>()) != cudaSuccess) return e;
    if ((e = configure_one<16, 8>()) != cudaSuccess) return e;
    if ((e = configure_one<8, 2>()) != cudaSuccess) return e;
    if ((e = configure_one<8, 4>()) != cudaSuccess) return e;
    if ((e = configure_one<4, 2>()) != cudaSuccess) return e;
    return configure_one<4, 4>();
}

// FP32, S in {4, 8, 16}
cudaError_t launch_group(const BatchArgs& a, int S, int B, int chunk, int sm_count, cudaStream_t stream) {
    if (S == 16 && B == 2) return launch_one<16, 2>(a, chunk, sm_count, stream);
    if (S == 16 && B == 4) return launch_one<16, 4>(a, chunk, sm_count, stream);
    if (S == 16 && B == 8) return launch_one<16, 8>(a, chunk, sm_count, stream);
    if (S == 8 && B == 2) return launch_one<8, 2>(a, chunk, sm_count, stream);
    if (S == 8 && B == 4) return launch_one<8, 4>(a, chunk, sm_count, stream);
    if (S == 4 && B == 2) return launch_one<4, 2>(a, chunk, sm_count, stream);
    if (S == 4 && B == 4) return launch_one<4, 4>(a, chunk, sm_count, stream);
    return cudaErrorNotSupported;
}

}  // namespace fsrk
