"""GB300 (sm_103a) hierarchical homogenization of segmented 3D images.

The compute path is the CUDA library libhh (csrc/, C ABI in include/hh.h);
this package only builds it and marshals arguments through ctypes
(`binding`). Nothing here computes on the CPU.
"""

from .binding import (Context, HHError, cnn_init_params, load, options, plan_partition,  # noqa: F401
                      surrogate_load, surrogate_save)
