"""Seeded synthetic inputs for correlation plenoptic imaging (CPI).

This package is input infrastructure shared by the tests, the benchmark and the
oracle checks.  It simulates the two detectors of a chaotic-light CPI set-up and
lays their frames out in memory; it contains none of the correlation or
refocusing arithmetic of the method itself.
"""

from .frames import (  # noqa: F401
    Acquisition,
    CONFIGS,
    batched_acquisitions,
    bin_file_frames,
    bin_file_layout,
    generate,
    model_maps,
    expected_gamma_counts,
    pack_bits_lsb,
    pack_side_by_side,
    random_gamma,
    uniform_planes,
)
from .model_init import DENOISER_PARAMS, denoiser_init  # noqa: F401,E402
