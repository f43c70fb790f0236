"""GB300-native Frequency Selective Reconstruction (FSR).

The hot path (weighting, 32 x 32 DFT, K x {argmax, damped coefficient update,
circular-shift residual update}, inverse and write-back) runs in hand-written
sm_103a CUDA kernels behind the C-ABI declared in ``include/fsr.h``.  This
package holds the thin ctypes binding over that library and the seeded input
generators.  Importing it does not load the CUDA library; the first call does.
"""
