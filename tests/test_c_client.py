"""The C ABI from plain C: tests/c_client/plan_info.c is compiled as C99 with
-Wall -Werror against include/qtam.h, linked against the in-tree libqtam.so,
and run; its host-only plan info (no GPU) must equal what the Python binding
and the oracle report for the same plan."""
import os
import shutil
import subprocess

import pytest

from oracle import qtam_oracle as O
from paper_2603_29785_gb300 import build as qbuild
from paper_2603_29785_gb300 import qtam

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def c_output(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = qtam.lib()                       # builds libqtam.so if it is missing or stale
    assert lib is not None
    libdir = os.path.dirname(qbuild.lib_path())
    exe = str(tmp_path_factory.mktemp("c_client") / "plan_info")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_client", "plan_info.c"),
           "-L", libdir, "-lqtam", f"-Wl,-rpath,{libdir}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    out = {}
    for line in r.stdout.splitlines():
        k, v = line.split(" ", 1)
        out[k] = v
    return out


def test_c_client_plan_info_matches_binding_and_oracle(c_output):
    p = qtam.Plan(4096.0, 262144, (4.0, 8.0, 16.0, 32.0, 64.0), 20.0, 2048.0, 128, device=-1)
    g = O.geometry(4096.0, 262144, (4.0, 8.0, 16.0, 32.0, 64.0), 20.0, 2048.0, 128)
    i = p.info
    for k in ("length", "n_bins", "n_planes", "rows_per_plane", "n_out", "h_max", "max_window",
              "envelope_bytes_per_segment", "band_bins", "kept_bins", "row_variant"):
        assert int(c_output[k]) == int(i[k]), k
    assert float(c_output["p_floor_rel"]) == i["p_floor_rel"]
    assert float(c_output["kappa"]) == i["kappa"]
    assert int(c_output["n_out"]) == g.M == 4800 and int(c_output["h_max"]) == g.h_max == 2346
    assert int(c_output["n_bins"]) == g.Nr


def test_c_client_sees_argument_errors(c_output):
    assert int(c_output["odd_length_status"]) == 1          # QTAM_ERR_INVALID_ARG
    assert c_output["odd_length_message"] == "yes"
    assert int(c_output["destroy"]) == 0


def _cuda_home():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime_api.h")):
            return cand
    return None


@pytest.mark.gpu
def test_c_client_forward_inverse_on_gpu(tmp_path):
    """forward + inverse driven from C (CUDA runtime C API buffers, default
    stream) against the FP64 oracle: FP32 tolerances 1e-6 (forward) and 1e-5
    (round trip against the projection)."""
    import numpy as np
    from paper_2603_29785_gb300 import synth
    cc, cuda = shutil.which("gcc") or shutil.which("cc"), _cuda_home()
    if cc is None or cuda is None:
        pytest.skip("no C compiler or CUDA headers")
    qtam.lib()
    libdir = os.path.dirname(qbuild.lib_path())
    exe = str(tmp_path / "roundtrip_gpu")
    cudalib = next((d for d in ("lib64", os.path.join("targets", "sbsa-linux", "lib"), "lib")
                    if os.path.exists(os.path.join(cuda, d, "libcudart.so"))), "lib64")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c_client", "roundtrip_gpu.c"),
           "-L", libdir, "-lqtam", "-L", os.path.join(cuda, cudalib), "-lcudart",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(cuda, cudalib)}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    N, B = 16384, 2
    x = np.stack([synth.white_sine_gaussian_segment(40 + b, n=N) for b in range(B)]).astype(np.float32)
    x.tofile(tmp_path / "x.bin")
    r = subprocess.run([exe, str(tmp_path / "x.bin"), str(tmp_path / "y.bin"), str(tmp_path / "xh.bin")],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    fields = r.stdout.split()
    M, P, K, tau = int(fields[1]), int(fields[3]), int(fields[5]), float(fields[7])
    g = O.geometry(4096.0, N, (8.0, 16.0), 20.0, 1024.0, 32)
    assert (M, P, K) == (g.M, g.P, g.K)
    Y = np.fromfile(tmp_path / "y.bin", dtype=np.complex64).reshape(B, P, K, M).astype(np.complex128)
    xh = np.fromfile(tmp_path / "xh.bin", dtype=np.float32).reshape(B, N).astype(np.float64)
    for b in range(B):
        ref = O.forward(g, x[b].astype(np.float64))
        assert np.linalg.norm(Y[b] - ref) / np.linalg.norm(ref) < 1e-6
        xp = O.projection(g, x[b].astype(np.float64), tau=tau)
        assert np.linalg.norm(xh[b] - xp) / np.linalg.norm(xp) < 1e-5
