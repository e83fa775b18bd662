"""GB300 (sm_103a) motion-blurred differentiable mesh renderer with the fast barycentric
coordinate solver of "Recovering 3D Shapes from Ultra-Fast Motion-Blurred Images"
(arXiv 2602.07860).  The compute path is the CUDA library ``libmbr.so`` (C ABI in
include/mbr.h); this package is its thin PyTorch binding."""
from .render import (Camera, Context, Motion, RenderBlur, camera_from_dict, default_context, mesh_tensors,
                     motion_from_dict, render_blur)

__all__ = ["Camera", "Context", "Motion", "RenderBlur", "camera_from_dict", "default_context", "mesh_tensors",
           "motion_from_dict", "render_blur"]
