"""GB300-native two-dimensional replica-exchange Wang-Landau sampling.

The sampling path (Wang-Landau trials, replica exchange, flatness checks,
iteration advance, merge/join/normalisation) runs in the CUDA kernels of
``librewl.so`` behind the C ABI of ``include/rewl.h``; :mod:`.rewl` is its
argument-marshalling binding.  Nothing is loaded at import time; the first
:class:`REWL` loads the library and fails loudly if it is missing.
"""
from .rewl import (F32, F32X2, FP64, JOIN_MARGINAL, JOIN_PER_SLICE, LNG_JOINED, LNG_MARGINAL_E,  # noqa: F401
                   PART_REST, PART_SAMPLE, PART_SAMPLE_PLAIN, REWL, SAMPLER_THREAD, SAMPLER_WARP, Batch, Config,
                   REWLError, TABLES_AUTO, TABLES_GLOBAL, TABLES_STAGED, LATTICE_AUTO,
                   LATTICE_REGISTER, LATTICE_SHARED, load_library, measure_peaks, philox,
                   relative_difference)
