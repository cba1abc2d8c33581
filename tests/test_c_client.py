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
