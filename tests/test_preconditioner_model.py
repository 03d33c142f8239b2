"""The sine-transform preconditioner of the Hartree CG (the library's default), modelled with
numpy/scipy on the oracle's 12th-order operator: its eigenvalues are those of the operator's
Toeplitz part, and it makes CG converge in a handful of iterations.  CPU only."""
import numpy as np
import pytest

from oracle import fd

scipy_fft = pytest.importorskip("scipy.fft")


def _lam1d(n, h):
    """-(a_0 + 2 sum_m a_m cos(m theta_k)) / h^2, theta_k = pi (k+1) / (n+1)."""
    a = fd.fd_coefficients()
    th = np.pi * (np.arange(n) + 1) / (n + 1)
    return -(a[0] + 2 * sum(a[m] * np.cos(m * th) for m in range(1, len(a)))) / h ** 2


def _apply_A(x, h):
    return -fd.laplacian(x, h)


def _precond(shape, h):
    lam = sum(_lam1d(n, h).reshape([n if i == ax else 1 for i in range(3)])
              for ax, n in enumerate(shape))
    return lambda r: scipy_fft.idstn(scipy_fft.dstn(r, type=1) / lam, type=1)


def test_sine_modes_are_eigenvectors_away_from_the_faces():
    # A sine mode of the zero-ghost operator: the rows farther than the stencil radius from
    # every face see the Toeplitz symbol exactly; rows nearer the faces differ.
    n, h, r = (30, 28, 26), 0.4, 6
    k = (3, 7, 11)
    z, y, x = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    mode = (np.sin(np.pi * (k[0] + 1) * (z + 1) / (n[0] + 1))
            * np.sin(np.pi * (k[1] + 1) * (y + 1) / (n[1] + 1))
            * np.sin(np.pi * (k[2] + 1) * (x + 1) / (n[2] + 1)))
    lam = sum(_lam1d(m, h)[kk] for m, kk in zip(n, k))
    Am = _apply_A(mode, h)
    inner = (slice(r, n[0] - r), slice(r, n[1] - r), slice(r, n[2] - r))
    assert np.max(np.abs(Am[inner] - lam * mode[inner])) < 1e-9 * lam
    assert np.max(np.abs(Am - lam * mode)) > 1e-6 * lam   # the face rows are not diagonal


@pytest.mark.parametrize("shape", [(24, 24, 24), (22, 16, 20)])
def test_pcg_converges_in_few_iterations(shape):
    h = 0.4
    rng = np.random.default_rng(5)
    b = rng.standard_normal(shape)
    M = _precond(shape, h)
    x = np.zeros(shape)
    r = b.copy()
    z = M(r)
    p = z.copy()
    rz = np.vdot(r, z)
    it = 0
    while np.linalg.norm(r) > 1e-12 * np.linalg.norm(b):
        Ap = _apply_A(p, h)
        al = rz / np.vdot(p, Ap)
        x += al * p
        r -= al * Ap
        z = M(r)
        rzn = np.vdot(r, z)
        p = z + (rzn / rz) * p
        rz = rzn
        it += 1
        assert it <= 10, it
    assert np.linalg.norm(b - _apply_A(x, h)) <= 2e-12 * np.linalg.norm(b)
