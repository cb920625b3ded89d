"""DeGraF detection + RLOF tracking (arXiv 1901.09971) as GB300 CUDA kernels.

The compute lives in libdegraf.so (C ABI, include/degraf.h); this package is the
thin torch binding. Nothing here computes on the CPU.
"""
from ._abi import (  # noqa: F401
    DegrafError, F16, F32, FB_REJECTED, MAXITER, OOB, PYR_APRON, SINGULAR, SMALL_EIG, TRACKED, load,
)
from .api import (  # noqa: F401
    BatchTracker, DeGraFDetect, DenseFlow, device_status, EpicParams, GmParams, HostPairTracker, PairTracker, RLOFTrack, RlofParams, build_pyramid, degraf_count, detect,
    detect_backward, epic_interpolate, epic_workspace_bytes, gm_workspace_bytes, pyramid_bytes, pyramid_layout, pyramid_planes, set_lanes, track,
    track_backward, track_fb, track_gm, track_pair, version,
)
