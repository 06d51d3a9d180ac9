"""Sparsity of the tableaux the kernels use (the coefficients live in
csrc/tableau.h): nonzeros per row of a~ and which b~_i are nonzero, and the
same for SSP3-IMEX(4,3,3) with its implicit part."""


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


def imex_structure():
    """SSP3-IMEX(4,3,3): per stage the nonzeros of the explicit row a~_i, of
    the implicit row a_i left of the diagonal, whether the stage's local
    operator is needed (b~_i != 0 or a later a~_ki != 0) and whether
    b~_i = b_i is nonzero.  Every diagonal a_ii is nonzero (alpha) and every
    stage's source is needed."""
    return dict(nnz_e=[0, 0, 1, 2], nnz_i=[0, 1, 1, 3], need_L=[False, True, True, True],
                b=[False, True, True, True])
