"""The row-FFT building blocks (csrc/fft_core.h) against numpy's FFT, on the CPU.

The shared-memory row transforms of the pruned 2-D FFT are made of in-register DFTs
(radix 2, 4, 8, 16), Stockham passes and the real/complex split.  The host program
tests/fft_core_check.cpp runs them with the device kernels' pass schedule; here the
results are compared with numpy.fft (complex forward/inverse, rfft, irfft * n).
"""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2407_03608_gb300", "csrc")


@pytest.fixture(scope="module")
def host_prog(tmp_path_factory):
    exe = tmp_path_factory.mktemp("fft") / "fft_core_check"
    # no floating-point contraction: the float-float steps rely on every product and sum
    # being rounded on its own
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                           os.path.join(ROOT, "tests", "fft_core_check.cpp"), "-o", str(exe)])
    return str(exe)


def run(host_prog, mode, L, data):
    inp = "%s %d\n" % (mode, L) + "\n".join("%.17g" % v for v in data) + "\n"
    out = subprocess.run([host_prog], input=inp, capture_output=True, text=True, check=True).stdout
    return np.array([float(v) for v in out.split()])


@pytest.mark.parametrize("L", [4, 5, 6, 7, 8, 9, 11, 12])
def test_complex_fft_both_directions(host_prog, L):
    n = 1 << L
    rng = np.random.default_rng(L)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    inter = np.column_stack([z.real, z.imag]).ravel()
    f = run(host_prog, "c2c", L, inter)
    got = f[0::2] + 1j * f[1::2]
    ref = np.fft.fft(z)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    b = run(host_prog, "ic2c", L, inter)
    got = b[0::2] + 1j * b[1::2]
    ref = np.fft.ifft(z) * n                      # unnormalised e^{+2 pi i}
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("L", [4, 5, 6, 7, 8, 12])
def test_first_pass_from_registers(host_prog, L):
    """The row kernels run the first pass on the elements each thread loaded from
    global memory (t + u N/16); the transform is unchanged."""
    n = 1 << L
    rng = np.random.default_rng(200 + L)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    f = run(host_prog, "c2cr", L, np.column_stack([z.real, z.imag]).ravel())
    got = f[0::2] + 1j * f[1::2]
    ref = np.fft.fft(z)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("L", [5, 8, 11, 12])
def test_float_passes(host_prog, L):
    """The passes in float (the FP32 plans' arithmetic) stay within a few float roundings
    of numpy's transform."""
    n = 1 << L
    rng = np.random.default_rng(300 + L)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    inter = np.column_stack([z.real, z.imag]).ravel()
    for mode, ref in (("fc2c", np.fft.fft(z)), ("fic2c", np.fft.ifft(z) * n)):
        f = run(host_prog, mode, L, inter)
        got = f[0::2] + 1j * f[1::2]
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 2e-6 * L, (mode, err)


@pytest.mark.parametrize("L", [4, 7, 10])
def test_real_split_matches_rfft_and_irfft(host_prog, L):
    n2 = 1 << L
    nf = 2 * n2
    rng = np.random.default_rng(100 + L)
    x = rng.standard_normal(nf)
    f = run(host_prog, "r2c", L, x)                  # x[2n], x[2n+1] pairs in order
    got = f[0::2] + 1j * f[1::2]
    ref = np.fft.rfft(x)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # inverse: a Hermitian half spectrum with modes above M zero (as after the mode box)
    M = int(0.4 * nf)
    X = np.zeros(n2 + 1, complex)
    X[:M + 1] = rng.standard_normal(M + 1) + 1j * rng.standard_normal(M + 1)
    X[0] = X[0].real
    inter = np.column_stack([X.real, X.imag]).ravel()
    y = run(host_prog, "c2r", L, inter)              # z[n] = x[2n] + i x[2n+1]
    ref = np.fft.irfft(X, nf) * nf                # unnormalised C2R
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("L", [5, 8, 12, 13])
def test_float_float_passes(host_prog, L):
    """The passes in float-float (the GP_DF64 plans' arithmetic, two float words a value)
    reach float64-grade accuracy: within 1e-13 of numpy's transform, elementwise relative
    to the largest output, where plain float stays near 1e-7."""
    n = 1 << L
    rng = np.random.default_rng(400 + L)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    inter = np.column_stack([z.real, z.imag]).ravel()
    for mode, ref in (("dc2c", np.fft.fft(z)), ("dic2c", np.fft.ifft(z) * n)):
        f = run(host_prog, mode, L, inter)
        got = f[0::2] + 1j * f[1::2]
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)), mode


@pytest.mark.parametrize("W,beta", [(9, 20.6), (13, 30.1), (16, 37.0)])
def test_float_float_kernel_values(host_prog, W, beta):
    """The exponential-of-semicircle kernel in float-float (sqrt_dd, exp_dd) against float64:
    within 5e-14 of psi(0) = 1 everywhere, and within 2e-13 relative where psi >= 1e-3 (near
    the ends of the support 1 - z^2 is formed with cancellation in either arithmetic)."""
    # the plans' offsets: xi = g - l0 with l0 = ceil(g - W/2), so xi in (W/2 - 1, W/2]
    rng = np.random.default_rng(W)
    j = rng.integers(0, W, 400)
    xi = W / 2.0 - rng.random(400)
    xi[:4] = W / 2.0 - np.array([0.0, 1e-12, 0.5, 1.0 - 1e-9])
    inp = "%.17g %d\n" % (beta, len(j)) + "\n".join("%d %.17g" % (a, b) for a, b in zip(j, xi)) + "\n"
    out = subprocess.run([host_prog], input="dpsi %d\n" % W + inp, capture_output=True, text=True,
                         check=True).stdout
    got = np.array([float(v) for v in out.split()])
    z = (j - xi) * 2.0 / W
    q = 1.0 - z * z
    ref = np.where(q > 0, np.exp(beta * (np.sqrt(np.maximum(q, 0.0)) - 1.0)), 0.0)
    inside = ref > 0
    assert np.all(got[~inside] == 0.0)
    assert np.max(np.abs(got - ref)) <= 5e-14
    big = ref >= 1e-3
    assert np.max(np.abs(got[big] - ref[big]) / ref[big]) <= 2e-13
