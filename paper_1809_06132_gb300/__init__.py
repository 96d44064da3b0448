"""GB300-native fisheye plane-sweep stereo and TSDF fusion (Cui et al.,
"Real-Time Dense Mapping for Self-Driving Vehicles using Fisheye Cameras").

The compute path is libpsweep.so (hand-written sm_103a CUDA kernels behind
the C ABI in include/psweep.h); this package is its thin Python binding.
"""
from .psweep import (EXPORTS, STATIC_MAX_BLOCKS, PsError, Sweep, Tsdf, load, lib_path, version, check_read,  # noqa: F401
                     Batch, Pipeline, SoftSweep, soft_depth, dense_fuse, se3_exp_left, batch_opts, batch_autotune, BATCH_SHORTEST_FIRST, BATCH_GIVEN_ORDER,
                     tsdf_integrate_dense_static,
                     PS_OK, PS_ERR_ARG, PS_ERR_OOM, PS_ERR_CAPACITY, PS_ERR_CUDA, PS_ERR_TIMEOUT, PS_ERR_STATE)
from ._build import build  # noqa: F401
