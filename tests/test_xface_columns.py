"""The column rule of the x-face traces at lane-group ends (x_col in
fr_device.cuh), checked on the host for many mesh shapes.

An element stores its low x face when its left neighbour (periodic along x)
is not the previous lane of its group of E elements, and its high face when
its right neighbour is not the next lane; the fused kernel reads exactly
those faces of the neighbours it cannot reach by a shuffle.  The rule must
give every stored face of one side a column of its own, below the row pitch
(a multiple of 32 at least the element count), and the reader must compute
the writer's column.  This restates the documented rule; the GPU tests run
the kernels on meshes of each kind (n_x < E, n_x a multiple of E, n_x > E
otherwise).
"""
import pytest


def x_col(e, E, mode, hi):
    if mode == 0:
        return e
    if mode == 1:
        return e // E
    inside = ((e + 1) % E != 0) if hi else (e % E != 0)
    return 2 * (e // E) + inside


def mode_for(nx, E):
    return 0 if nx < E else (1 if nx % E == 0 else 2)


def on_chip(e_left, e_right, E):
    return e_right == e_left + 1 and e_right % E != 0


@pytest.mark.parametrize("E", [4, 8, 16, 32])
@pytest.mark.parametrize("nx,nrest", [(1, 3), (3, 5), (7, 2), (16, 3), (31, 2), (32, 3),
                                      (33, 2), (40, 3), (47, 1), (64, 2), (67, 3), (84, 2),
                                      (96, 1), (168, 1)])
def test_stored_x_faces_have_their_own_columns(E, nx, nrest):
    ne = nx * nrest
    stride = (ne + 31) // 32 * 32
    mode = mode_for(nx, E)
    cols = {False: {}, True: {}}
    for e in range(ne):
        ex, row = e % nx, e // nx
        left = row * nx + (ex - 1) % nx
        right = row * nx + (ex + 1) % nx
        for hi, stored in ((False, not on_chip(left, e, E)), (True, not on_chip(e, right, E))):
            if not stored:
                continue
            c = x_col(e, E, mode, hi)
            assert 0 <= c < stride, (e, hi, c, stride)
            assert c not in cols[hi], (e, cols[hi].get(c), hi, c)
            cols[hi][c] = e
    # the reader: each element whose neighbour is off-lane reads that
    # neighbour's face at the column the writer used
    for e in range(ne):
        ex, row = e % nx, e // nx
        left = row * nx + (ex - 1) % nx
        right = row * nx + (ex + 1) % nx
        if not on_chip(left, e, E):
            assert cols[True][x_col(left, E, mode, True)] == left
        if not on_chip(e, right, E):
            assert cols[False][x_col(right, E, mode, False)] == right
