"""Test-side plain assembly of Q1 systems in numpy (dense), written
independently of the C oracle, for brute-force pins on tiny grids."""
import numpy as np

KREF = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0


def stiffness(a2d):
    """Dense stiffness over all (nx+1)(ny+1) nodes of a rectangle of
    elements with coefficient a2d[ny][nx]."""
    ny, nx = a2d.shape
    N = (nx + 1) * (ny + 1)
    A = np.zeros((N, N))
    for ey in range(ny):
        for ex in range(nx):
            idx = [ey * (nx + 1) + ex, ey * (nx + 1) + ex + 1,
                   (ey + 1) * (nx + 1) + ex + 1, (ey + 1) * (nx + 1) + ex]
            A[np.ix_(idx, idx)] += a2d[ey, ex] * KREF
    return A


def boundary_mask(nx, ny):
    m = np.zeros((ny + 1, nx + 1), dtype=bool)
    m[0, :] = m[-1, :] = True
    m[:, 0] = m[:, -1] = True
    return m.reshape(-1)


def bilinear(nx, ny):
    """The four bilinear nodal functions of the rectangle, [4][N]."""
    X, Y = np.meshgrid(np.arange(nx + 1) / nx, np.arange(ny + 1) / ny)
    return np.stack([(1 - X) * (1 - Y), X * (1 - Y), X * Y, (1 - X) * Y]).reshape(4, -1)


def harmonic_extension(a2d, g):
    """Solve the Dirichlet problem with boundary values g (full nodal
    vector, interior entries ignored) by a dense library solve."""
    ny, nx = a2d.shape
    A = stiffness(a2d)
    bd = boundary_mask(nx, ny)
    it = ~bd
    u = g.copy()
    u[it] = np.linalg.solve(A[np.ix_(it, it)], -A[np.ix_(it, bd)] @ g[bd])
    return u
