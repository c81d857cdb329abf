"""Dense-matrix builder for tiny lattices (test helper)."""
import numpy as np


def dense(apply, shape):
    """Matrix of a linear map on arrays of ``shape`` (column j = apply(e_j)).

    The output may have a different size from the input (rectangular maps).
    """
    n = int(np.prod(shape))
    cols = []
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        cols.append(np.asarray(apply(e.reshape(shape))).reshape(-1).copy())
        e[j] = 0.0
    return np.stack(cols, axis=1)
