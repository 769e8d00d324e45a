"""Semi-implicit Fourier spectral step (the paper's spectral solver scheme, Sec.
"Construction of Semi-Implicit Fourier Spectral Scheme"): linear terms are
integrated implicitly in Fourier space, nonlinear terms explicitly in real
space.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: plain numpy (the FFT is
numpy's), FP64, no code shared with the GPU library.

Readings (the paper names the scheme and its references but prints no
splitting):
  * the Laplacian is the continuous symbol -|k|^2 with k = 2 pi m / (n h) per
    axis (a spectral method, not a stencil);
  * every linear term is implicit, the cubic term explicit:
      Allen-Cahn    phi_t = lap phi + c1 phi - c2 phi^3
                    L(k) = c1 - |k|^2,            N = -c2 phi^3
      Cahn-Hilliard phi_t = lap(c2 phi^3 - c1 phi - kappa lap phi)
                    L(k) = |k|^2 (c1 - kappa |k|^2), N^ = -|k|^2 c2 (phi^3)^
    and one step is  phi^_{n+1} = (phi^_n + dt N^(phi_n)) / (1 - dt L(k));
  * the step is defined while 1 - dt L(k) > 0 for every k (Allen-Cahn
    dt c1 < 1, Cahn-Hilliard dt c1^2 / (4 kappa) < 1).
Fields are numpy arrays in (ny, nx) or (nz, ny, nx) order, x fastest; the real
FFT runs along x.
"""
import numpy as np

AC, CH = 0, 1


def k_squared(shape, h: float) -> np.ndarray:
    """|k|^2 on the real-FFT half spectrum of a grid of numpy ``shape``."""
    axes = []
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            k = 2.0 * np.pi * np.fft.rfftfreq(n, d=h)
        else:
            k = 2.0 * np.pi * np.fft.fftfreq(n, d=h)
        axes.append(k)
    mesh = np.meshgrid(*axes, indexing="ij")
    return sum(k * k for k in mesh)


def linear_symbol(model: int, k2: np.ndarray, c1: float, kappa: float) -> np.ndarray:
    if model == AC:
        return c1 - k2
    return k2 * (c1 - kappa * k2)


def stable(model: int, dt: float, c1: float, kappa: float) -> bool:
    """1 - dt L(k) > 0 for every k (the bound of the reading above)."""
    if model == AC:
        return dt * c1 < 1.0
    return kappa > 0 and dt * c1 * c1 / (4.0 * kappa) < 1.0


def step(model: int, u, *, h: float = 1.0, dt: float, c1: float = 1.0, c2: float = 1.0, kappa: float = 1.0,
         nsteps: int = 1) -> np.ndarray:
    """``nsteps`` semi-implicit spectral steps from ``u`` (a copy is returned)."""
    u = np.array(u, dtype=np.float64, copy=True)
    shape = u.shape
    axes = tuple(range(u.ndim))
    k2 = k_squared(shape, h)
    denom = 1.0 - dt * linear_symbol(model, k2, c1, kappa)
    uh = np.fft.rfftn(u, axes=axes)
    for _ in range(nsteps):
        cube = (u * u) * u
        if model == AC:
            nh = np.fft.rfftn(-c2 * cube, axes=axes)
        else:
            nh = -k2 * np.fft.rfftn(c2 * cube, axes=axes)
        uh = (uh + dt * nh) / denom
        u = np.fft.irfftn(uh, s=shape, axes=axes)
    return u
