/*
 * Plain FP64 CPU oracle for Frequency Selective Reconstruction (FSR).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline leg of the benchmark.  Nothing in the product path links it.
 *
 * Every routine follows the paper's steps in the paper's order and notation,
 * without blocking, fusion or reordering:
 *   Sec. II   Eq. (2)  sampled signal f~ (f on the known set, 0 elsewhere)
 *             Eq. (5)  spatial weighting w
 *             Eq. (7)  R_w^(0) = F2{ f~ . w }
 *             Eq. (8)  (u,v) = argmax_(k,l) w_f[k,l] |R_w[k,l]|^2
 *             Eq. (9)  frequency weighting w_f
 *             Eq. (10) p = R_w[u,v] / W[0,0]
 *             Eq. (11) G[u,v] += gamma p S^2
 *             Eq. (12) R_w[k,l] -= gamma p W[k-u, l-v]  for all (k,l)
 *             then g = IDFT2(G), f^ = f~ on known pixels, g elsewhere
 *   Sec. III-A Eq. (13) N = ceil(Y/B) ceil(X/B) independent blocks
 *   Sec. III-A Eqs. (14)-(15) the circular indices i, j of W[k-u, l-v]
 *
 * Readings where the paper is silent (each repeated at its use):
 *   - DFT sign and scale: forward e^{-j...} unnormalised, inverse 1/S^2 e^{+j...};
 *   - argmax ties go to the lowest linear index k*S + l (strict '>' scan);
 *   - the output is Re g (single complex components are updated, Eq. 11);
 *   - pixels outside the image are unknown; a block without a known pixel
 *     keeps g = 0 and skips its iterations (its W[0,0] is 0);
 *   - the weight centre for even S is (S-1)/2.
 *
 * Build with -ffp-contract=off so every product is rounded on its own: the
 * twiddle table is exactly conjugate-symmetric, hence the spectrum of a real
 * block is exactly Hermitian and conjugate-pair ties are exact.
 */
#include "fsr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

/* Twiddles T[t] = e^{-j 2 pi t / S}.  Computed for t <= S/2 and mirrored so
 * that T[S-t] = conj(T[t]) holds bit for bit; the points on the axes take
 * their exact values (1, -j, -1, +j). */
static void twiddles(int S, double *Tre, double *Tim)
{
    for (int t = 0; t <= S / 2; ++t) {
        double a = TWO_PI * (double)t / (double)S;
        Tre[t] = cos(a);
        Tim[t] = -sin(a);
    }
    Tre[0] = 1.0;
    Tim[0] = 0.0;
    if (S % 2 == 0) {
        Tre[S / 2] = -1.0;
        Tim[S / 2] = 0.0;
    }
    if (S % 4 == 0) {
        Tre[S / 4] = 0.0;
        Tim[S / 4] = -1.0;
    }
    for (int t = S / 2 + 1; t < S; ++t) {
        Tre[t] = Tre[S - t];
        Tim[t] = -Tim[S - t];
    }
}

/* Eq. (5) without the restriction to known pixels. */
void fsr_oracle_spatial_weight(int S, double rho, double *w0)
{
    double c = (double)(S - 1) / 2.0;  /* reading: centre of an even support */
    for (int m = 0; m < S; ++m)
        for (int n = 0; n < S; ++n) {
            double dm = (double)m - c, dn = (double)n - c;
            w0[m * S + n] = pow(rho, sqrt(dm * dm + dn * dn));
        }
}

/* Eq. (9): w_f = (1 - sqrt(2) sqrt(kt^2/S^2 + lt^2/S^2))^2,
 * kt = S/2 - |k - S/2|, lt = S/2 - |l - S/2|. */
void fsr_oracle_freq_weight(int S, double *wf)
{
    double half = (double)S / 2.0;
    for (int k = 0; k < S; ++k)
        for (int l = 0; l < S; ++l) {
            double kt = half - fabs((double)k - half);
            double lt = half - fabs((double)l - half);
            double r = sqrt(kt * kt / ((double)S * S) + lt * lt / ((double)S * S));
            double b = 1.0 - sqrt(2.0) * r;
            wf[k * S + l] = b * b;
        }
}

/* X[k,l] = sum_m e^{-j2pi km/S} ( sum_n x[m,n] e^{-j2pi ln/S} ): the DFT
 * definition with the double sum written as nested sums. */
void fsr_oracle_dft2_real(int S, const double *x, double *Xre, double *Xim)
{
    double *Tre = malloc(sizeof(double) * S), *Tim = malloc(sizeof(double) * S);
    double *Yre = malloc(sizeof(double) * S * S), *Yim = malloc(sizeof(double) * S * S);
    twiddles(S, Tre, Tim);
    for (int m = 0; m < S; ++m)
        for (int l = 0; l < S; ++l) {
            double sr = 0.0, si = 0.0;
            for (int n = 0; n < S; ++n) {
                int t = (l * n) % S;
                sr += x[m * S + n] * Tre[t];
                si += x[m * S + n] * Tim[t];
            }
            Yre[m * S + l] = sr;
            Yim[m * S + l] = si;
        }
    for (int k = 0; k < S; ++k)
        for (int l = 0; l < S; ++l) {
            double sr = 0.0, si = 0.0;
            for (int m = 0; m < S; ++m) {
                int t = (k * m) % S;
                double a = Tre[t], b = Tim[t];
                double c = Yre[m * S + l], d = Yim[m * S + l];
                sr += a * c - b * d;
                si += a * d + b * c;
            }
            Xre[k * S + l] = sr;
            Xim[k * S + l] = si;
        }
    free(Tre); free(Tim); free(Yre); free(Yim);
}

/* One support block: Eqs. (2), (5)-(12) in order.  scale[i] multiplies the
 * weight of Eq. (5) at pixel i: 1 on the known set K of Eq. (2), 0 on
 * unknown pixels, and in the re-use form of fsr_oracle_image_reuse the
 * re-use weight delta on pixels reconstructed by earlier blocks (reading:
 * those pixels join the set of Eq. 2 with the weight delta rho^dist). */
int fsr_oracle_block_scaled(const fsr_oracle_params *P, const double *f,
                            const double *scale, fsr_oracle_block_out *o)
{
    if (!P || !f || !scale || P->S <= 0 || P->K < 0) return -1;
    const int S = P->S, K = P->K, SS = S * S;
    int skipped = 0;

    double *w0 = malloc(sizeof(double) * SS), *wf = malloc(sizeof(double) * SS);
    double *w = malloc(sizeof(double) * SS), *x = malloc(sizeof(double) * SS);
    double *Rre = malloc(sizeof(double) * SS), *Rim = malloc(sizeof(double) * SS);
    double *Wre = malloc(sizeof(double) * SS), *Wim = malloc(sizeof(double) * SS);
    double *Gre = calloc(SS, sizeof(double)), *Gim = calloc(SS, sizeof(double));

    fsr_oracle_spatial_weight(S, P->rho, w0);
    if (P->freq_weight) {
        fsr_oracle_freq_weight(S, wf);
    } else {
        for (int i = 0; i < SS; ++i) wf[i] = 1.0;
    }

    /* Eqs. (2), (5), (6): w = w0 on known pixels (scale 1), 0 elsewhere;
     * the weighted sampled signal f~ . w.  Unknown values are never read. */
    for (int i = 0; i < SS; ++i) {
        w[i] = scale[i] > 0.0 ? scale[i] * w0[i] : 0.0;
        x[i] = scale[i] > 0.0 ? f[i] * w[i] : 0.0;
    }
    /* Eq. (7) and the weighting spectrum W = F2{w}. */
    fsr_oracle_dft2_real(S, x, Rre, Rim);
    fsr_oracle_dft2_real(S, w, Wre, Wim);
    const double W0 = Wre[0];

    if (o && o->w) memcpy(o->w, w, sizeof(double) * SS);
    if (o && o->R0re) memcpy(o->R0re, Rre, sizeof(double) * SS);
    if (o && o->R0im) memcpy(o->R0im, Rim, sizeof(double) * SS);
    if (o && o->Wre) memcpy(o->Wre, Wre, sizeof(double) * SS);
    if (o && o->Wim) memcpy(o->Wim, Wim, sizeof(double) * SS);
    if (o && o->Rhre) memcpy(o->Rhre, Rre, sizeof(double) * SS);
    if (o && o->Rhim) memcpy(o->Rhim, Rim, sizeof(double) * SS);

    /* Reading: a block without a known pixel has W[0,0] = 0 and Eq. (10) is
     * undefined; the model stays G = 0. */
    int any_known = 0;
    for (int i = 0; i < SS; ++i) any_known |= (scale[i] > 0.0);
    if (!any_known) skipped = 1;

    for (int nu = 0; nu < K; ++nu) {
        if (skipped) {
            if (o && o->seq) o->seq[nu] = -1;
            if (o && o->pre) o->pre[nu] = 0.0;
            if (o && o->pim) o->pim[nu] = 0.0;
            if (o && o->margin) o->margin[nu] = 0.0;
            if (o && o->margin_nc) o->margin_nc[nu] = 0.0;
            if (o && o->Rhre) memcpy(o->Rhre + (size_t)(nu + 1) * SS, Rre, sizeof(double) * SS);
            if (o && o->Rhim) memcpy(o->Rhim + (size_t)(nu + 1) * SS, Rim, sizeof(double) * SS);
            continue;
        }
        if (P->conj_pairs) {
            /* Ablation, not the paper's Eqs. (11)-(12): the real-valued model
             * of the original FSR.  The basis pair phi_uv + its conjugate
             * phi_{-u,-v} is added with the coefficients a = gamma p and a*
             * (p of Eq. 10), so G stays Hermitian and g real:
             *   G[u,v] += a S^2,  G[-u,-v] += a* S^2,
             *   R_w[k,l] -= a W[k-u, l-v] + a* W[k+u, l+v]
             * (the residual update of Eq. 12 applied to both basis images).
             * A self-conjugate (u,v) (2u = 2v = 0 mod S) is one real basis
             * image and takes the single update.  R_w stays Hermitian, so the
             * members of a pair tie: the scan visits the member with the
             * lower linear index only, which also keeps the margin meaningful.
             * The sums and differences of the two W entries make the update of
             * (-k,-l) the exact conjugate of that of (k,l). */
            double top = -1.0, runner = -1.0;
            int sel = 0;
            for (int k = 0; k < S; ++k)
                for (int l = 0; l < S; ++l) {
                    const int lin = k * S + l, lin_conj = ((S - k) % S) * S + (S - l) % S;
                    if (lin_conj < lin) continue;
                    const double ob = wf[lin] * (Rre[lin] * Rre[lin] + Rim[lin] * Rim[lin]);
                    if (ob > top) {
                        runner = top;
                        top = ob;
                        sel = lin;
                    } else if (ob > runner) {
                        runner = ob;
                    }
                }
            const int su = sel / S, sv = sel % S;
            const int sel_conj = ((S - su) % S) * S + (S - sv) % S;
            const double qre = Rre[sel] / W0, qim = Rim[sel] / W0;      /* Eq. (10) */
            const double cre = P->gamma * qre, cim = P->gamma * qim;    /* a = gamma p */
            Gre[sel] += cre * (double)SS;
            Gim[sel] += cim * (double)SS;
            if (sel_conj != sel) {
                Gre[sel_conj] += cre * (double)SS;
                Gim[sel_conj] -= cim * (double)SS;
            }
            for (int k = 0; k < S; ++k)
                for (int l = 0; l < S; ++l) {
                    const int d1 = ((k + S - su) % S) * S + (l + S - sv) % S;   /* W[k-u, l-v] */
                    const int d2 = ((k + su) % S) * S + (l + sv) % S;           /* W[k+u, l+v] */
                    double ur, ui;
                    if (sel_conj == sel) {
                        ur = cre * Wre[d1] - cim * Wim[d1];
                        ui = cre * Wim[d1] + cim * Wre[d1];
                    } else {
                        const double sr = Wre[d1] + Wre[d2], si = Wim[d1] + Wim[d2];
                        const double dr = Wre[d1] - Wre[d2], di = Wim[d1] - Wim[d2];
                        ur = cre * sr - cim * di;    /* Re(a W1 + a* W2) */
                        ui = cre * si + cim * dr;    /* Im(a W1 + a* W2) */
                    }
                    Rre[k * S + l] -= ur;
                    Rim[k * S + l] -= ui;
                }
            if (o && o->seq) o->seq[nu] = sel;
            if (o && o->pre) o->pre[nu] = qre;
            if (o && o->pim) o->pim[nu] = qim;
            if (o && o->margin) o->margin[nu] = top > 0.0 ? (top - runner) / top : 0.0;
            if (o && o->margin_nc) o->margin_nc[nu] = top > 0.0 ? (top - runner) / top : 0.0;
            if (o && o->Rhre) memcpy(o->Rhre + (size_t)(nu + 1) * SS, Rre, sizeof(double) * SS);
            if (o && o->Rhim) memcpy(o->Rhim + (size_t)(nu + 1) * SS, Rim, sizeof(double) * SS);
            continue;
        }
        /* Eq. (8): exhaustive scan; strict '>' keeps the lowest index on ties. */
        double best = -1.0, second = -1.0;
        int idx = 0;
        for (int i = 0; i < SS; ++i) {
            double obj = wf[i] * (Rre[i] * Rre[i] + Rim[i] * Rim[i]);
            if (obj > best) {
                second = best;
                best = obj;
                idx = i;
            } else if (obj > second) {
                second = obj;
            }
        }
        const int u = idx / S, v = idx % S;
        if (o && o->margin_nc) {   /* diagnostic: the runner-up other than the conjugate of (u,v) */
            const int cj = ((S - u) % S) * S + (S - v) % S;
            double second_nc = -1.0;
            for (int i = 0; i < SS; ++i) {
                if (i == idx || i == cj) continue;
                const double ob = wf[i] * (Rre[i] * Rre[i] + Rim[i] * Rim[i]);
                if (ob > second_nc) second_nc = ob;
            }
            o->margin_nc[nu] = best > 0.0 ? (best - second_nc) / best : 0.0;
        }

        /* Eq. (10): p = R_w[u,v] / W[0,0]. */
        const double pre = Rre[idx] / W0, pim = Rim[idx] / W0;
        /* Eq. (11): G[u,v] += gamma p S^2. */
        Gre[idx] += P->gamma * pre * (double)SS;
        Gim[idx] += P->gamma * pim * (double)SS;

        /* Eq. (12) with the circular indices of Eqs. (14)-(15). */
        const double are = P->gamma * pre, aim = P->gamma * pim;
        for (int k = 0; k < S; ++k) {
            int i = (k - u >= 0) ? k - u : S + k - u;
            for (int l = 0; l < S; ++l) {
                int j = (l - v >= 0) ? l - v : S + l - v;
                double c = Wre[i * S + j], d = Wim[i * S + j];
                Rre[k * S + l] -= are * c - aim * d;
                Rim[k * S + l] -= are * d + aim * c;
            }
        }

        if (o && o->seq) o->seq[nu] = idx;
        if (o && o->pre) o->pre[nu] = pre;
        if (o && o->pim) o->pim[nu] = pim;
        if (o && o->margin) o->margin[nu] = best > 0.0 ? (best - second) / best : 0.0;
        if (o && o->Rhre) memcpy(o->Rhre + (size_t)(nu + 1) * SS, Rre, sizeof(double) * SS);
        if (o && o->Rhim) memcpy(o->Rhim + (size_t)(nu + 1) * SS, Rim, sizeof(double) * SS);
    }

    if (o && o->Gre) memcpy(o->Gre, Gre, sizeof(double) * SS);
    if (o && o->Gim) memcpy(o->Gim, Gim, sizeof(double) * SS);

    /* g = IDFT2(G): g[m,n] = 1/S^2 sum_{k,l} G[k,l] e^{+j2pi(km+ln)/S}. */
    if (o && (o->gre || o->gim)) {
        double *Tre = malloc(sizeof(double) * S), *Tim = malloc(sizeof(double) * S);
        twiddles(S, Tre, Tim);
        for (int m = 0; m < S; ++m)
            for (int n = 0; n < S; ++n) {
                if (o->g_need && !o->g_need[m * S + n]) {
                    if (o->gre) o->gre[m * S + n] = NAN;
                    if (o->gim) o->gim[m * S + n] = NAN;
                    continue;
                }
                double sr = 0.0, si = 0.0;
                for (int k = 0; k < S; ++k)
                    for (int l = 0; l < S; ++l) {
                        int t = (k * m + l * n) % S;
                        double c = Tre[t], d = -Tim[t];  /* e^{+j theta} = conj(T) */
                        double a = Gre[k * S + l], b = Gim[k * S + l];
                        sr += a * c - b * d;
                        si += a * d + b * c;
                    }
                if (o->gre) o->gre[m * S + n] = sr / (double)SS;
                if (o->gim) o->gim[m * S + n] = si / (double)SS;
            }
        free(Tre); free(Tim);
    }

    free(w0); free(wf); free(w); free(x); free(Rre); free(Rim);
    free(Wre); free(Wim); free(Gre); free(Gim);
    return skipped;
}

/* The paper's block routine: weight w0 on the known set, 0 elsewhere. */
int fsr_oracle_block(const fsr_oracle_params *P, const double *f,
                     const unsigned char *known, fsr_oracle_block_out *o)
{
    if (!P || !f || !known || P->S <= 0 || P->K < 0) return -1;
    const int SS = P->S * P->S;
    double *scale = malloc(sizeof(double) * SS);
    for (int i = 0; i < SS; ++i) scale[i] = known[i] ? 1.0 : 0.0;
    int r = fsr_oracle_block_scaled(P, f, scale, o);
    free(scale);
    return r;
}

int fsr_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sec. III-A: every B x B target block b = by*nbx + bx is reconstructed on its
 * own support, origin (by*B - L, bx*B - L), by the block routine above. */
long fsr_oracle_image_blocks(const float *img, const unsigned char *mask,
                             int H, int Wd, int pitch, int B, int L,
                             const fsr_oracle_params *P, long nsel,
                             const long *block_ids, int nthreads,
                             double *out_target, double *out_im, int *seq, double *margin,
                             double *margin_nc)
{
    if (!img || !mask || !P || !out_target || H <= 0 || Wd <= 0 || pitch < Wd ||
        B <= 0 || L < 0 || P->S != B + 2 * L || P->K < 0)
        return -1;
    const int S = P->S, K = P->K;
    const long nbx = (Wd + B - 1) / B, nby = (H + B - 1) / B;
    if (!block_ids) nsel = nbx * nby;
    long n_empty = 0;
    int bad = 0;
    if (nthreads <= 0) nthreads = fsr_oracle_max_threads();

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads) reduction(+ : n_empty) reduction(| : bad)
#endif
    for (long s = 0; s < nsel; ++s) {
        const long b = block_ids ? block_ids[s] : s;
        if (b < 0 || b >= nbx * nby) { bad = 1; continue; }
        const long by = b / nbx, bx = b % nbx;
        const long y0 = by * B - L, x0 = bx * B - L;
        double *f = malloc(sizeof(double) * S * S);
        unsigned char *kn = malloc((size_t)S * S);
        double *gre = malloc(sizeof(double) * S * S);
        double *gim = out_im ? malloc(sizeof(double) * S * S) : NULL;
        unsigned char *need = calloc((size_t)S * S, 1);
        for (int a = 0; a < B; ++a)
            for (int c = 0; c < B; ++c) need[(L + a) * S + (L + c)] = 1;
        for (int m = 0; m < S; ++m)
            for (int n = 0; n < S; ++n) {
                long y = y0 + m, x = x0 + n;
                int inside = (y >= 0 && y < H && x >= 0 && x < Wd);  /* reading: outside = unknown */
                int k = inside && mask[y * pitch + x] != 0;
                kn[m * S + n] = (unsigned char)k;
                f[m * S + n] = k ? (double)img[y * pitch + x] : 0.0;
            }
        fsr_oracle_block_out o;
        memset(&o, 0, sizeof o);
        o.seq = seq ? seq + s * K : NULL;
        o.margin = margin ? margin + s * K : NULL;
        o.margin_nc = margin_nc ? margin_nc + s * K : NULL;
        o.gre = gre;
        o.gim = gim;      /* diagnostic: Im g (the model is complex, Eq. 11) */
        o.g_need = need;  /* only the target pixels are written back */
        int r = fsr_oracle_block(P, f, kn, &o);
        if (r < 0) bad = 1;
        if (r == 1) n_empty += 1;
        /* Write-back: known pixels keep f, unknown ones take Re g. */
        for (int a = 0; a < B; ++a)
            for (int c = 0; c < B; ++c) {
                int m = L + a, n = L + c;
                long y = y0 + m, x = x0 + n;
                double val;
                if (y >= H || x >= Wd) val = NAN;
                else val = kn[m * S + n] ? f[m * S + n] : gre[m * S + n];
                out_target[(s * B + a) * B + c] = val;
                if (out_im)
                    out_im[(s * B + a) * B + c] =
                        (y >= H || x >= Wd) ? NAN : (kn[m * S + n] ? 0.0 : gim[m * S + n]);
            }
        free(f); free(kn); free(gre); free(gim); free(need);
    }
    return bad ? -1 : n_empty;
}

/* Re-use of reconstructed pixels: the sequential form of the original FSR,
 * which the paper leaves out in Sec. II for the sake of parallelism.
 * Readings (the paper does not define this form):
 *   - blocks are processed one after the other in line-scan (raster) order
 *     b = by*nbx + bx;
 *   - when block b runs, an unknown pixel of the target of an earlier block
 *     (b' < b) holds that block's reconstruction Re g and takes part in the
 *     support of b with the weight delta rho^dist (delta: the re-use weight);
 *     unknown pixels of later blocks stay unknown;
 *   - everything else is the paper's block routine; delta = 0 gives the
 *     independent blocks of fsr_oracle_image_blocks.
 * out: H x Wd (row pitch Wd) reconstruction of blocks 0 .. nblocks-1 (known
 * pixels copied, NaN on pixels of later blocks); nblocks <= 0: all blocks.
 * seq, margin: optional nblocks*K.  Single-threaded (each block depends on
 * the ones before it).
 * given: optional H x Wd reconstruction (row pitch Wd) to take the re-used
 * values from instead of the routine's own earlier results; each block then
 * depends on `given` only and the blocks run in parallel (nthreads).  With
 * given = the routine's own result every block sees the same support as in
 * the sequential run.
 * Returns the number of blocks without any known or re-used pixel, or -1 on
 * error. */
long fsr_oracle_image_reuse(const float *img, const unsigned char *mask,
                            int H, int Wd, int pitch, int B, int L,
                            const fsr_oracle_params *P, double delta, long nblocks,
                            const double *given, int nthreads,
                            double *out, int *seq, double *margin)
{
    if (!img || !mask || !P || !out || H <= 0 || Wd <= 0 || pitch < Wd ||
        B <= 0 || L < 0 || P->S != B + 2 * L || P->K < 0 || !(delta >= 0.0 && delta <= 1.0))
        return -1;
    const int S = P->S, K = P->K;
    const long nbx = (Wd + B - 1) / B, nby = (H + B - 1) / B;
    if (nblocks <= 0 || nblocks > nbx * nby) nblocks = nbx * nby;
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < Wd; ++x)
            out[y * Wd + x] = mask[y * pitch + x] ? (double)img[y * pitch + x] : NAN;
    const double *src = given ? given : out;   /* where re-used values come from */
    long n_empty = 0;
    int bad = 0;
    if (nthreads <= 0) nthreads = fsr_oracle_max_threads();
    if (!given) nthreads = 1;                    /* the sequential form */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads) reduction(+ : n_empty) reduction(| : bad)
#endif
    for (long b = 0; b < nblocks; ++b) {
        if (bad) continue;
        double *f = malloc(sizeof(double) * S * S), *scale = malloc(sizeof(double) * S * S);
        double *gre = malloc(sizeof(double) * S * S);
        unsigned char *need = calloc((size_t)S * S, 1);
        for (int a = 0; a < B; ++a)
            for (int c = 0; c < B; ++c) need[(L + a) * S + (L + c)] = 1;
        const long by = b / nbx;          /* raster order: block row, then column */
        const long bx = b - by * nbx;
        const long y0 = by * B - L;       /* support origin (Sec. III-A) */
        const long x0 = bx * B - L;
        for (int m = 0; m < S; ++m)
            for (int n = 0; n < S; ++n) {
                const long y = y0 + m, x = x0 + n;
                double v = 0.0, sc = 0.0;
                if (y >= 0 && y < H && x >= 0 && x < Wd) {      /* reading: outside = unknown */
                    if (mask[y * pitch + x]) {
                        v = (double)img[y * pitch + x];
                        sc = 1.0;
                    } else if ((y / B) * nbx + (x / B) < b) {    /* reconstructed by an earlier block */
                        v = src[y * Wd + x];
                        sc = delta;
                    }
                }
                f[m * S + n] = v;
                scale[m * S + n] = sc;
            }
        fsr_oracle_block_out o;
        memset(&o, 0, sizeof o);
        o.seq = seq ? seq + b * K : NULL;
        o.margin = margin ? margin + b * K : NULL;
        o.gre = gre;
        o.g_need = need;
        int r = fsr_oracle_block_scaled(P, f, scale, &o);
        if (r < 0) bad = 1;
        if (r == 1) n_empty += 1;
        /* write-back of the target: unknown pixels take Re g */
        for (int a = 0; a < B; ++a)
            for (int c = 0; c < B; ++c) {
                const long y = y0 + L + a, x = x0 + L + c;
                if (y < H && x < Wd && !mask[y * pitch + x]) out[y * Wd + x] = gre[(L + a) * S + (L + c)];
            }
        free(f); free(scale); free(gre); free(need);
    }
    return bad ? -1 : n_empty;
}
