"""GB300-native RadiusFPS: exact farthest point sampling with spherical-voxel pruning.

The compute path is librfps.so (hand-written sm_103a CUDA behind the C ABI of
include/rfps.h); this package is its thin Python binding plus the batching,
autotuning and serving layers around it.
"""

from . import autotune, batch, serve, shard  # noqa: F401
from ._lib import (  # noqa: F401
    Counters,
    Index,
    Opts,
    RfpsError,
    batch_workspace_size,
    bandwidth_probe,
    counters,
    fps,
    fps_batched,
    fps_host,
    host_workspace_size,
    launch_count,
    lib,
    plain_fps,
    plain_fps_batched,
    plain_workspace_size,
    resolved_opts,
    status,
    sync_floor,
    workspace_size,
)
