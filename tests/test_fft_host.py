"""The shared-memory FFT passes of the CUDA path (fft.cuh), emulated thread by thread
on the CPU in barrier order, against a direct DFT in double precision.  No GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("src", ["fft_emul.cpp", "fft_regs_emul.cpp"])
def test_fft_passes_match_direct_dft(tmp_path, src):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "fft"
    subprocess.run([gxx, "-O2", "-std=c++17", "-include", "array", os.path.join(HERE, "cpp", src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    sizes = dict(zip(out[0::2], map(float, out[1::2])))
    assert set(sizes) == {"512", "1024", "2048", "4096", "8192"}
    for m, err in sizes.items():
        assert err < 5e-7, (m, err)    # FP32 transform vs double: ~1e-7 relative


def test_fft384_matches_direct_dft(tmp_path):
    """The 384-point transform (3 x 128) of the paper reverb's frames: an impulse, a
    single complex exponential and two noise inputs against the direct DFT."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "fft384"
    subprocess.run([gxx, "-O2", "-std=c++17", os.path.join(HERE, "cpp", "fft384_emul.cpp"), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    errs = [float(x) for x in out.stdout.split()[1::2]]
    assert len(errs) == 4, out.stdout
    assert max(errs) < 5e-7, errs
    assert out.returncode == 0
