"""The separable row form of the isotropic D3Q27 gradient, as the row-blocked
stencil passes of the CUDA path evaluate it (nine neighbour rows, weights
W(0) = 4, W(+-1) = 1 over 72, four nodes per thread reading each row as
x0-1 .. x0+4), equals the oracle's 26-point sum of Sec. 4.1 on periodic grids
and under the walls' mirror rule (Phi_x odd).  A check of the derivation on
the CPU; the kernels themselves are held to the oracle by the GPU parity
tests."""

import numpy as np
import pytest

import oracle as O


def _rows_form(phi, alpha, walls=False, odd=False, V=4):
    nz, ny, nx = phi.shape
    flat = phi.ravel()
    out = np.zeros(flat.size)
    for n0 in range(0, flat.size, V):
        x0 = n0 % nx
        t = n0 // nx
        y, z = t % ny, t // ny
        pl = nx * ny
        xm = (0 if walls else nx - 1) if x0 == 0 else x0 - 1
        xp = (nx - 1 if walls else 0) if x0 + V == nx else x0 + V
        ys = [(ny - 1 if y == 0 else y - 1) * nx, y * nx, (0 if y == ny - 1 else y + 1) * nx]
        zs = [(nz - 1 if z == 0 else z - 1) * pl, z * pl, (0 if z == nz - 1 else z + 1) * pl]
        d = np.zeros(V)
        for cz in (-1, 0, 1):
            for cy in (-1, 0, 1):
                rb = zs[cz + 1] + ys[cy + 1]
                v = np.concatenate([[flat[rb + xm]], flat[rb + x0:rb + x0 + V], [flat[rb + xp]]])
                if odd and walls and x0 == 0:
                    v[0] = -v[0]
                if odd and walls and x0 + V == nx:
                    v[-1] = -v[-1]
                Wy, Wz = (1 if cy else 4), (1 if cz else 4)
                for j in range(V):
                    if alpha == 0:
                        d[j] += Wy * Wz * (v[j + 2] - v[j])
                    else:
                        s = v[j] + 4 * v[j + 1] + v[j + 2]
                        d[j] += (cy * Wz if alpha == 1 else cz * Wy) * s
        own = zs[1] + ys[1] + x0
        out[own:own + V] = d / 72.0
    return out.reshape(phi.shape)


@pytest.mark.parametrize("shape", [(3, 5, 8), (2, 2, 4), (3, 4, 12)])
@pytest.mark.parametrize("walls,odd", [(False, False), (True, False), (True, True)])
def test_row_form_equals_the_26_point_gradient(shape, walls, odd):
    phi = np.random.Generator(np.random.PCG64(sum(shape))).standard_normal(shape)
    for alpha in range(3):
        ref = O.iso_derivative(phi, alpha, walls_x=walls, odd_x=odd and alpha == 0)
        got = _rows_form(phi, alpha, walls=walls, odd=odd and alpha == 0)
        np.testing.assert_allclose(got, ref, atol=1e-14)
