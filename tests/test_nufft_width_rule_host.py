"""The NUFFT discretisation the host selector picks (App. D; the exponential-of-semicircle
kernel psi(z) = exp(beta (sqrt(1 - z^2) - 1)) over `width` cells with beta = 0.97 pi
width (1 - 1/(2 sigma)), sigma = nf / (2M + 1)) reaches the requested nufft_tol.

A plain type-1 NUFFT written here on the CPU (periodic spreading onto the nf-cell grid
of period 1/dw, numpy's FFT, division by the kernel's transform from Gauss-Legendre
quadrature) with the selector's nf, width and beta is compared with the oracle's exact
non-uniform DFT.  No GPU; the CUDA kernels are not involved.
"""
import numpy as np
import pytest

import gpinputs
from oracle import nudft


def es_type1(x, c, M, dw, nf, width, beta):
    """f_n = sum_j c_j exp(-2 pi i n dw x_j), |n| <= M, through the spreading kernel."""
    P = 1.0 / dw
    h = P / nf
    half = width / 2.0
    grid = np.zeros(nf)
    for xj, cj in zip(x, c):
        t = xj / h
        k = np.arange(int(np.ceil(t - half)), int(np.ceil(t - half)) + width + 1)
        z = (k - t) / half
        inside = np.abs(z) <= 1.0
        np.add.at(grid, k[inside] % nf, cj * np.exp(beta * (np.sqrt(1.0 - z[inside] ** 2) - 1.0)))
    n = np.arange(-M, M + 1)
    U = np.fft.fft(grid)[n % nf]
    zq, wq = np.polynomial.legendre.leggauss(400)
    psi = np.exp(beta * (np.sqrt(1.0 - zq ** 2) - 1.0))
    psihat = half * h * (np.cos(np.pi * n[:, None] * width * zq[None, :] / nf) * psi * wq).sum(axis=1)
    return h * U / psihat


@pytest.fixture(scope="module")
def abi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03608_gb300 import abi
    return abi


@pytest.mark.parametrize("tol,upsamp,nf", [(1e-4, 1.25, None), (1e-7, 2.0, None), (1e-10, 1.25, None),
                                           (1e-12, 2.0, None), (1e-4, None, 728), (1e-7, None, 728),
                                           (1e-9, None, 728), (1e-7, None, 1164), (1e-9, None, 1164)])
def test_selected_kernel_reaches_the_tolerance(abi, tol, upsamp, nf):
    set_bits = abi.GP_SET_NUFFT | (abi.GP_SET_NF if nf else 0)
    o = abi.default_opts(precision=abi.GP_FP64, nufft_tol=tol, upsampfac=upsamp or 2.0, nf=nf or 0, set=set_bits,
                         param_mode=abi.GP_PARAMS_PAPER)
    i = abi.gp_plan_params(1, 300, 1.5, 1e-3, 0.01, 0.03, [0.0], [1.0], o)
    M, width = int(i["M"]), int(i["kernel_width"])
    assert i["upsampfac"] == pytest.approx(i["nf"] / (2 * M + 1))
    assert i["kernel_beta"] == pytest.approx(0.97 * np.pi * width * (1 - 1 / (2 * i["upsampfac"])))
    w = gpinputs.config_1d(300)
    x = w.points[:, 0]
    c = np.random.default_rng(1).standard_normal(300)
    got = es_type1(x, c, M, i["dw"], int(i["nf"]), width, i["kernel_beta"])
    exact = nudft.type1(x[:, None], c[None, :], M, i["dw"])[0]
    err = float(np.linalg.norm(got - exact) / np.linalg.norm(exact))
    assert err <= tol, (err, width, i["upsampfac"])
    # one cell narrower would not be enough in the tighter cases (the rule is not wasteful)
    if tol <= 1e-7:
        beta1 = 0.97 * np.pi * (width - 1) * (1 - 1 / (2 * i["upsampfac"]))
        narrow = es_type1(x, c, M, i["dw"], int(i["nf"]), width - 1, beta1)
        assert np.linalg.norm(narrow - exact) / np.linalg.norm(exact) > tol / 30
