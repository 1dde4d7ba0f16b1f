"""Shared helpers of the GPU tests: the library build, oracle caches, error metrics.

Tolerances (written in each test): FP64 GPU form relative L2 <= 1e-12 against the FP64
oracle; FP32 forms <= 1e-5.
"""
import functools

import numpy as np

TOL_FP64 = 1e-12
TOL_FP32 = 1e-5


@functools.lru_cache(maxsize=None)
def library():
    from paper_1904_07400_gb300 import build, native
    build.build()
    return native.load()


@functools.lru_cache(maxsize=8)
def oracle_solver(nx, ny, k, dx, dy, G=1.0):
    from oracle.convolution import Solver
    return Solver(nx, ny, k, dx, dy, G)


def rel_l2_pair(fx, fy, rx, ry):
    from oracle.norms import rel_l2
    return rel_l2(fx, fy, rx, ry)


def to_np(t):
    return t.detach().double().cpu().numpy()
