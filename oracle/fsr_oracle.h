/*
 * Plain FP64 CPU oracle for Frequency Selective Reconstruction (FSR),
 * frequency-domain form of Regensky et al., "Real-Time Frequency Selective
 * Reconstruction through Register-Based Argmax Calculation" (MMSP 2020),
 * Sec. II, Eqs. (1)-(12), with the block tiling of Sec. III-A, Eq. (13).
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only callers.  The product (CUDA)
 * path shares no code, header, table or helper with this file.
 *
 * Conventions (readings of the paper, each stated where it is used):
 *   - arrays are row-major S x S, index [m*S + n] in space and [k*S + l] in
 *     frequency; k pairs with the row index m, l with the column index n;
 *   - forward DFT is unnormalised with e^{-j 2 pi (k m + l n) / S}, inverse
 *     carries 1/S^2 and e^{+j ...} (forced by the S^2 factor of Eq. (11));
 *   - argmax ties go to the lowest linear index k*S + l;
 *   - pixels outside the image are unknown.
 */
#ifndef FSR_ORACLE_H
#define FSR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int S;            /* support size S = B + 2L */
    int K;            /* number of iterations (paper: fixed count, Sec. II) */
    double rho;       /* spatial decay factor rho-hat, Eq. (5) */
    double gamma;     /* orthogonality deficiency compensation, Eqs. (11)-(12) */
    int freq_weight;  /* 1: objective w_f |R_w|^2 (Eq. 8); 0: |R_w|^2 */
    int conj_pairs;   /* 0: the paper's single complex component per iteration
                         (Eqs. 11-12); 1: ablation, the selected component and
                         its conjugate together (a real model, see the .c file) */
} fsr_oracle_params;

/* Optional per-block outputs; any pointer may be NULL. */
typedef struct {
    double *w;        /* S*S spatial weighting w[m,n], Eq. (5) */
    double *R0re;     /* S*S initial weighted residual spectrum, Eq. (7) */
    double *R0im;
    double *Wre;      /* S*S spectrum of the weighting, W = F2{w} */
    double *Wim;
    int    *seq;      /* K selected indices u*S + v (Eq. 8); -1 when skipped */
    double *pre;      /* K projection coefficients p, Eq. (10) */
    double *pim;
    double *margin;   /* K relative gaps (best - second) / best of the objective */
    double *margin_nc; /* K relative gaps (best - second) / best with the conjugate of the
                          selected component left out of "second" (diagnostic: ties
                          between components that are not a conjugate pair) */
    double *Rhre;     /* (K+1)*S*S residual spectrum before each iteration */
    double *Rhim;
    double *Gre;      /* S*S final model spectrum G, Eq. (11) */
    double *Gim;
    double *gre;      /* S*S final model g = IDFT2(G) (complex) */
    double *gim;
    const unsigned char *g_need; /* S*S flags: evaluate g only there (NULL: all) */
} fsr_oracle_block_out;

/* w0[m*S+n] = rho^sqrt((m-c)^2 + (n-c)^2), c = (S-1)/2  (Eq. 5, all pixels). */
void fsr_oracle_spatial_weight(int S, double rho, double *w0);

/* wf[k*S+l] per Eq. (9). */
void fsr_oracle_freq_weight(int S, double *wf);

/* X = F2{x} for a real S x S input by the DFT definition. */
void fsr_oracle_dft2_real(int S, const double *x, double *Xre, double *Xim);

/* FSR on one support block.  f: S*S support values (only known ones are
 * read); known: S*S flags (nonzero = sampled, the set K of Eq. 2).
 * Returns 1 when the block has no known pixel (iterations skipped, g = 0),
 * 0 otherwise, -1 on bad arguments. */
int fsr_oracle_block(const fsr_oracle_params *P, const double *f,
                     const unsigned char *known, fsr_oracle_block_out *o);

/* The block routine with a weight scale per pixel: w = scale * w0 (Eq. 5),
 * pixels with scale 0 are unknown (the set K of Eq. 2 is {scale > 0}).
 * fsr_oracle_block is this routine with scale = 1 on known pixels, 0 else. */
int fsr_oracle_block_scaled(const fsr_oracle_params *P, const double *f,
                            const double *scale, fsr_oracle_block_out *o);

/* FSR over selected blocks of an image (Sec. III-A tiling).
 * img/mask: H x Wd, row pitch in elements; mask nonzero = known.
 * Block b = by * nbx + bx with nbx = ceil(Wd/B), nby = ceil(H/B).
 * block_ids: nsel indices, or NULL for all blocks in order (nsel = nbx*nby).
 * out_target: nsel*B*B reconstructed target pixels (NaN outside the image).
 * out_im: optional nsel*B*B diagnostic, Im g at the unknown target pixels
 *         (0 at known ones, NaN outside the image); the output is Re g.
 * seq, margin, margin_nc: nsel*K each, optional.
 * nthreads: OpenMP threads (<= 0: library default).
 * Returns the number of blocks without any known pixel, or -1 on error. */
long fsr_oracle_image_blocks(const float *img, const unsigned char *mask,
                             int H, int Wd, int pitch, int B, int L,
                             const fsr_oracle_params *P, long nsel,
                             const long *block_ids, int nthreads,
                             double *out_target, double *out_im, int *seq, double *margin,
                             double *margin_nc);

/* Re-use of reconstructed pixels (the sequential form the paper leaves out,
 * Sec. II): blocks in raster order; unknown pixels of earlier blocks' targets
 * enter later supports with their reconstruction and the weight
 * delta * rho^dist.  out: H x Wd reconstruction of the first nblocks blocks
 * (<= 0: all; NaN on unknown pixels of later blocks); seq, margin optional
 * (nblocks*K).  given: optional H x Wd reconstruction the re-used values are
 * taken from instead (each block then depends on it alone; nthreads OpenMP
 * threads, <= 0: default).  Returns the number of blocks without any known
 * or re-used pixel, or -1 on error. */
long fsr_oracle_image_reuse(const float *img, const unsigned char *mask,
                            int H, int Wd, int pitch, int B, int L,
                            const fsr_oracle_params *P, double delta, long nblocks,
                            const double *given, int nthreads,
                            double *out, int *seq, double *margin);

/* Number of OpenMP threads the image routine would use by default. */
int fsr_oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
