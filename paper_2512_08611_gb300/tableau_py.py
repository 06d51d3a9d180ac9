"""Sparsity of the explicit tableaux the kernels use (the coefficients live in
csrc/tableau.h): nonzeros per row of a~ and which b~_i are nonzero."""


def stages_nnz_b(N):
    if N == 0:
        return [0], [True]
    if N == 1:
        return [0, 1], [True, True]
    if N == 2:
        return [0, 1, 2], [True, True, True]
    if N == 3:
        return [0, 1, 1, 1], [True, True, True, True]
    if N == 4:
        return [0, 1, 2, 2, 2, 5], [True, False, True, True, True, True]
    raise ValueError(N)
