"""Plain FP64 CPU oracle for Frequency Selective Reconstruction.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` import it.  The product path never does.
"""
from .oracle import (  # noqa: F401
    build,
    spatial_weight,
    freq_weight,
    dft2_real,
    fsr_block,
    fsr_image_blocks,
    fsr_image_reuse,
    assemble_image,
    max_threads,
    default,
    build_variant,
    source_text,
    OracleLib,
)
