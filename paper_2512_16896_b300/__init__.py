"""Sceniris hot path on B300: Python binding of libsceniris_b300.so.

The binding only marshals arguments: it turns torch CUDA tensors into device
pointers and fills the C structs declared in include/sceniris.h. Every step of
the path runs in the library's CUDA kernels; there is no CPU or eager-PyTorch
fallback. If the shared library is missing or fails to load, import of the
native handle raises.
"""
from ._native import (  # noqa: F401
    LIB_PATH,
    SceniError,
    Context,
    DeviceBatch,
    CollideConfig,
    lib,
    sample_poses,
    sample_parts,
    collide,
    collide_last_work,
    collide_last_tri_work,
    ik_last_work,
    generate,
    ik_reach,
    ik_dls_step,
    make_arm,
    ik_params,
    Surrogate,
    ReachMap,
    RMAP_DEFAULT,
    train_params,
    order_by_work,
)
