"""Random coefficient fields and rotations for the synthetic problems."""
import numpy as np


def gaussian_random_field(shape, corr_len, sigma, rng):
    """Stationary Gaussian field with covariance sigma^2 exp(-(r/corr_len)^2).

    White noise N(0,1) on a grid padded by 3*corr_len on every side is convolved,
    axis by axis, with the kernel exp(-2 x^2 / corr_len^2) truncated at 3*corr_len
    (self-convolution of that kernel is exp(-x^2/corr_len^2)); the interior is then
    normalised to unit sample standard deviation and scaled by sigma.
    Returned array has `shape`, with axis 0 = x (fastest in the flat ordering
    used elsewhere, i.e. callers flatten with order='F').
    """
    pad = int(np.ceil(3 * corr_len))
    big = tuple(s + 2 * pad for s in shape)
    w = rng.standard_normal(big)
    t = np.arange(-pad, pad + 1, dtype=np.float64)
    ker = np.exp(-2.0 * t * t / (corr_len * corr_len))
    for ax in range(len(shape)):
        w = np.apply_along_axis(lambda v: np.convolve(v, ker, mode="same"), ax, w)
    sl = tuple(slice(pad, pad + s) for s in shape)
    f = w[sl]
    f = f - f.mean()
    f = f / f.std()
    return sigma * f


def rotation_2d(deg):
    a = np.deg2rad(deg)
    return np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])


def rotation_zyx(az, ay, ax):
    """Intrinsic z-y-x Euler rotation R = Rz(az) Ry(ay) Rx(ax), angles in degrees."""
    a, b, c = np.deg2rad([az, ay, ax])
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Ry = np.array([[np.cos(b), 0, np.sin(b)], [0, 1, 0], [-np.sin(b), 0, np.cos(b)]])
    Rx = np.array([[1, 0, 0], [0, np.cos(c), -np.sin(c)], [0, np.sin(c), np.cos(c)]])
    return Rz @ Ry @ Rx
