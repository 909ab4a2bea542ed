"""GB300-native pair-cascade particle-in-cell library (arXiv:2012.05587).

The compute path is ``libcascade.so`` (hand-written CUDA for sm_103a); this
package loads it, marshals arguments through the C ABI of
``include/cascade.h`` and uses PyTorch only for device memory and streams.
"""
from .capi import (  # noqa: F401
    CASCADE_FP32_MIXED, CASCADE_FP64, CascadeError, cascade_counts, cascade_create,
    cascade_create_from_state, cascade_destroy, cascade_diag, cascade_footprint, cascade_gauss,
    cascade_particles, cascade_step, cascade_sync, load, use_torch_allocator,
)
from .cascade import Cascade, CascadeBatch  # noqa: F401
