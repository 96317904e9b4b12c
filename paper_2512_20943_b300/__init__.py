"""AirGS splatting path on B300 (sm_103a): a C-ABI CUDA library (libairgs.so)
with a thin PyTorch binding.

    rast = Rasterizer()
    rast.set_anchor(means, log_scales, quats, opacity_logit, sh)
    rast.apply_frame_update(update_map, lo, hi)          # Sec. II Eq. 3, Sec. III-B/C
    out = rast.render(cams, save=True)                   # tile splatting forward
    loss, grads = rast.render_backward_l1(out.state, target)

The library is required: there is no CPU fallback.
"""
from ._abi import (AIRGS_DELTA_ANCHOR, AIRGS_DELTA_PREV, AIRGS_QUAT_ADD, LIB_PATH, load_library)
from .rasterizer import (AirGSError, RasterConfig, RasterizeGaussians, Rasterizer, RenderResult, RenderState,
                         camera_array, camera_struct, image_sizes, rasterize, split_views)

__all__ = [
    "AIRGS_DELTA_ANCHOR", "AIRGS_DELTA_PREV", "AIRGS_QUAT_ADD", "LIB_PATH", "load_library", "AirGSError",
    "RasterConfig", "RasterizeGaussians", "Rasterizer", "RenderResult", "RenderState", "camera_array",
    "camera_struct", "image_sizes", "rasterize", "split_views",
]
