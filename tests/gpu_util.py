"""Helpers shared by the GPU tests: build the CUDA library and open a context."""
import functools

import numpy as np


@functools.lru_cache(maxsize=1)
def ctx():
    from paper_1309_4018_b300.build import build
    build()
    from paper_1309_4018_b300 import pbbem
    return pbbem.Context(0)


def problem(d, **params):
    from paper_1309_4018_b300 import pbbem
    pb = pbbem.Problem.from_dict(ctx(), d)
    pb.setup(**params)
    return pb


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
