"""FCFS (Fully Convolutional Fractional Scaling, arXiv 2203.10670) on GB300.

libfcfs (C ABI, include/fcfs.h) holds the hand-written sm_103a kernels; this
package is its Python binding.  Build with ``paper_2203_10670_gb300.build.build()``.
"""
from .fcfs import (BICUBIC, BILINEAR, FCFS, NEAREST, PAD_CONSTANT, PAD_REFLECT, PAD_REPLICATE, Axis, FCFSFunction,
                   fcfs_backward, fcfs_backward_workspace, fcfs_clear_plans, fcfs_device_status, fcfs_forward, fcfs_geometry,
                   fcfs_make_weights, fcfs_tune_forward, make_desc, resize, resize_backward, Server, FCFSFull2d,
                   FCFSFull2dFunction, make_desc_full2d, resize_full2d, resize_full2d_backward, resize_fused,
                   fcfs_forward_fused, ACT_NONE, ACT_RELU, ACT_LEAKY_RELU, ACT_CLAMP)

__all__ = ["FCFS", "FCFSFunction", "FCFSFull2d", "FCFSFull2dFunction", "resize_full2d", "resize_full2d_backward",
           "make_desc_full2d", "resize_fused", "fcfs_forward_fused", "ACT_NONE", "ACT_RELU",
           "ACT_LEAKY_RELU", "ACT_CLAMP", "Server", "Axis", "resize", "resize_backward", "make_desc", "fcfs_make_weights",
           "fcfs_geometry", "fcfs_forward", "fcfs_backward", "fcfs_backward_workspace", "fcfs_tune_forward",
           "fcfs_clear_plans", "fcfs_device_status", "NEAREST", "BILINEAR", "BICUBIC", "PAD_REPLICATE", "PAD_CONSTANT", "PAD_REFLECT"]
