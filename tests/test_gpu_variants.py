"""Every row-kernel variant (runtime engine and each compile-time launch
shape) computes the same transform: forward envelopes and the inverse
accumulation are checked against the FP64 oracle for every envelope length
the variants are built for."""
import numpy as np
import pytest

from oracle import qtam_oracle as O
from paper_2603_29785_gb300 import qtam, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (fs, N, qs, fmin, fmax, K) -> envelope length M
GEOMS = {
    4800: (4096.0, 262144, (4.0, 8.0, 16.0, 32.0, 64.0), 20.0, 2048.0, 128),
    2400: (4096.0, 131072, (8.0, 16.0, 32.0), 20.0, 2048.0, 128),
    1200: (4096.0, 65536, (8.0, 16.0, 32.0), 20.0, 2048.0, 128),
    600: (4096.0, 32768, (8.0, 16.0, 32.0), 20.0, 2048.0, 128),
    500: (4096.0, 16384, (8.0, 16.0), 20.0, 1024.0, 32),
    300: (4096.0, 16384, (8.0, 16.0, 32.0), 20.0, 2048.0, 128),
    150: (4096.0, 8192, (8.0, 16.0, 32.0), 20.0, 2048.0, 128),
    75: (4096.0, 4096, (8.0, 16.0, 32.0), 20.0, 2048.0, 128),
    8192: (4096.0, 262144, (4.0, 8.0, 16.0, 32.0, 64.0), 20.0, 2048.0, 128, 8192),   # n_out = 8192
}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("M", sorted(GEOMS))
def test_every_variant_matches_oracle(M):
    fs, N, qs, fmin, fmax, K = GEOMS[M][:6]
    n_out = GEOMS[M][6] if len(GEOMS[M]) > 6 else 0
    p = qtam.Plan(fs, N, qs, fmin, fmax, K, n_out=n_out, device=0)
    assert p.M == M
    g = O.geometry(fs, N, qs, fmin, fmax, K, n_out=n_out)
    variants = qtam.qtam_plan_variants(p.handle)
    assert variants[0] == -1 and len(variants) >= 2, variants
    x = synth.glitchy_segment(M, N, fs, chirp=True).astype(np.float64)
    X = O.spectrum(x)
    rows = [(a, k) for a in range(g.P) for k in (0, 1, K // 3, K // 2, K - 2, K - 1)]
    Yref = {(a, k): O.forward_row(g, X, a, k) for a, k in rows}
    big = max(np.max(np.abs(v)) for v in Yref.values())
    B = 2                                    # second segment checks the segment offset
    Xd = torch.from_numpy(np.stack([X, 0.5 * X]).astype(np.complex64)).cuda()
    rng = synth.rng(M)
    Yin = (rng.standard_normal((g.P, g.K, g.M)) + 1j * rng.standard_normal((g.P, g.K, g.M)))
    Aref = O.accumulate(g, Yin)
    Yd = torch.from_numpy(np.stack([Yin, -Yin]).astype(np.complex64)).cuda()
    for v in variants:
        qtam.qtam_plan_set_variant(p.handle, v)
        y = p.envelopes(Xd)
        A = p.accumulate(Yd)
        torch.cuda.synchronize()
        Y = y.cpu().numpy().astype(np.complex128)
        An = A.cpu().numpy().astype(np.complex128)
        name = qtam.qtam_variant_describe(v)["name"]
        for a, k in rows:
            assert rel(Y[0, a, k], Yref[a, k]) < 1e-6, (name, a, k)
            assert np.max(np.abs(Y[0, a, k] - Yref[a, k])) <= 1e-5 * big, (name, a, k)
            assert rel(Y[1, a, k], 0.5 * Yref[a, k]) < 1e-6, (name, a, k)
        assert rel(An[0], Aref) < 1e-6, name
        assert rel(An[1], -Aref) < 1e-6, name


@pytest.mark.parametrize("N", [2048, 4096, 8192, 16384, 32768, 65536, 131072, 262144, 524288])
def test_synthesis_stage_large(N):
    fs = 4096.0
    p = qtam.Plan(fs, N, (8.0,), 30.0, 1000.0, 16, max_window_hz=20.0, device=0)
    g = O.geometry(fs, N, (8.0,), 30.0, 1000.0, 16, max_window_hz=20.0)
    Y = O.forward(g, synth.white(5, N))
    A = O.accumulate(g, Y)
    x = p.synthesize(torch.from_numpy(A[None].astype(np.complex64)).cuda())
    torch.cuda.synchronize()
    ref = O.inverse(g, Y, tau=p.info["p_floor_rel"])
    assert rel(x.cpu().numpy()[0].astype(np.float64), ref) < 1e-5
