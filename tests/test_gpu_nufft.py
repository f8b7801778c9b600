"""The standalone NUFFTs (wave1d_nufft_*) against the oracle's direct sums.

type-1 S_k = (1/2 pi) sum_j c_j e^{+ikx_j} (eq. densco) and type-2 u_j = sum_{|k|<=K} alpha_k
e^{-ikx_j} (eq. historySol1), in FP64 (kernel weights precomputed) and in mixed precision (FP32
kernel Chebyshev series, moments and sums in FP32 with the dominant terms compensated, FP64 FFT).
Error: max |gpu - direct| / max |direct|
over the whole output.  Bars: FP64 at tol 1e-12 -> 1e-10 (the plan's NUFFT accuracy); mixed at tol
1e-6 -> 1e-6 (the mixed mode's stated accuracy).  At M = 1e6 (the clustered periodic workload)
the direct sums are taken at sampled modes and points.
"""
import numpy as np
import pytest

from oracle import wfp
from paper_2507_07823_gb300 import build, wave1d, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wave1d.lib()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _inputs(M, K, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-np.pi, np.pi, M)
    c = rng.uniform(0.5, 1.5, M) * np.where(rng.uniform(size=M) < 0.8, 1.0, -1.0)
    decay = 1.0 / (1.0 + np.arange(K + 1) / 300.0)
    alpha = (rng.standard_normal(K + 1) + 1j * rng.standard_normal(K + 1)) * decay
    alpha[0] = alpha[0].real
    return x, c, alpha


def _run(nu, c, alpha):
    import torch
    K = nu.K
    cd = torch.tensor(c[nu.perm], dtype=torch.float64, device="cuda")
    Sd = torch.zeros(2 * (K + 1), dtype=torch.float64, device="cuda")
    ad = torch.tensor(np.stack([alpha.real, alpha.imag], 1).reshape(-1), dtype=torch.float64, device="cuda")
    ud = torch.zeros(nu.M, dtype=torch.float64, device="cuda")
    nu.type1(cd, Sd)
    nu.type2(ad, ud)
    torch.cuda.synchronize()
    S = Sd.cpu().numpy()
    u = np.empty(nu.M)
    u[nu.perm] = ud.cpu().numpy()
    return S[0::2] + 1j * S[1::2], u


@pytest.mark.parametrize("precision,tol,bar", [(0, 1e-12, 1e-10), (1, 1e-6, 1e-6)])
def test_nufft_against_direct_sums(precision, tol, bar):
    """M = 3000 random points, K = 3141 (the dt = 1e-3 mode count), both transforms, twice."""
    M, K = 3000, 3141
    x, c, alpha = _inputs(M, K, 2507)
    nu = wave1d.Nufft(x, K, tol, precision)
    try:
        S, u = _run(nu, c, alpha)
        S2, u2 = _run(nu, c, alpha)
    finally:
        nu.close()
    assert np.array_equal(S, S2) and np.array_equal(u, u2)          # deterministic
    eS, eu = _rel(S, wfp.type1(c, x, K)), _rel(u, wfp.type2(alpha, x))
    print(f"precision {precision} tol {tol}: type-1 {eS:.2e} type-2 {eu:.2e}")
    assert eS < bar and eu < bar
    if precision == 1:
        assert nu.kernel_err < 3e-7


def test_nufft_small_and_ragged():
    """M = 1 and M = 37 (not a multiple of any block), a point on the box edge, K = 5."""
    for M in (1, 37):
        x, c, alpha = _inputs(M, 5, 11 + M)
        x[0] = -np.pi
        for precision, tol, bar in ((0, 1e-12, 1e-10), (1, 1e-6, 1e-6)):
            nu = wave1d.Nufft(x, 5, tol, precision)
            try:
                S, u = _run(nu, c, alpha)
            finally:
                nu.close()
            assert _rel(S, wfp.type1(c, x, 5)) < bar and _rel(u, wfp.type2(alpha, x)) < bar


def test_nufft_clustered_million_points_sampled():
    """The M = 1e6 clustered periodic workload (16 Gaussians sigma 0.05 + 20% uniform), K = 6283:
    type-1 at 48 sampled modes and type-2 at 400 sampled points against the direct sums, FP64
    (tol 1e-10) and mixed (tol 1e-6)."""
    w = W.config2()
    K = int(np.floor(np.pi / w.dt))
    rng = np.random.default_rng(7)
    c = rng.uniform(0.5, 1.5, w.M)
    alpha = (rng.standard_normal(K + 1) + 1j * rng.standard_normal(K + 1)) / (1.0 + np.arange(K + 1) / 300.0)
    alpha[0] = alpha[0].real                  # alpha_{-k} = conj(alpha_k) makes alpha_0 real
    ks = np.sort(rng.choice(K + 1, 48, replace=False))
    js = rng.choice(w.M, 400, replace=False)
    S_ref = np.array([np.sum(c * np.exp(1j * k * w.x)) for k in ks]) / (2 * np.pi)
    u_ref = wfp.type2(alpha, w.x[js])
    for precision, tol, bar in ((0, 1e-10, 1e-8), (1, 1e-6, 1e-6)):
        nu = wave1d.Nufft(w.x, K, tol, precision)
        try:
            S, u = _run(nu, c, alpha)
        finally:
            nu.close()
        eS = float(np.max(np.abs(S[ks] - S_ref)) / np.max(np.abs(S_ref)))
        eu = _rel(u[js], u_ref)
        print(f"M=1e6 precision {precision}: type-1 {eS:.2e} type-2 {eu:.2e}")
        assert eS < bar and eu < bar


def test_nufft_dense_cells_and_wrap():
    """Runs longer than a spreading unit: 6000 points within 1e-9 of one position, 3000 in a second
    cell, 2000 straddling the periodic seam at -pi / +pi, 1000 uniform; K = 400."""
    rng = np.random.default_rng(99)
    x = np.concatenate([1.234 + 1e-9 * rng.standard_normal(6000),
                        -0.5 + 1e-4 * rng.uniform(size=3000),
                        np.pi - 1e-3 * rng.uniform(size=1000),
                        -np.pi + 1e-3 * rng.uniform(size=1000),
                        rng.uniform(-np.pi, np.pi, 1000)])
    M, K = x.size, 400
    c = rng.uniform(0.5, 1.5, M) * np.where(rng.uniform(size=M) < 0.7, 1.0, -1.0)
    alpha = (rng.standard_normal(K + 1) + 1j * rng.standard_normal(K + 1)) / (1.0 + np.arange(K + 1) / 50.0)
    alpha[0] = alpha[0].real
    S_ref, u_ref = wfp.type1(c, x, K), wfp.type2(alpha, x)
    for precision, tol, bar in ((0, 1e-12, 1e-10), (1, 1e-6, 1e-6)):
        nu = wave1d.Nufft(x, K, tol, precision)
        try:
            S, u = _run(nu, c, alpha)
        finally:
            nu.close()
        eS, eu = _rel(S, S_ref), _rel(u, u_ref)
        print(f"dense cells precision {precision}: type-1 {eS:.2e} type-2 {eu:.2e}")
        assert eS < bar and eu < bar


def test_nufft_mixed_needs_tol_1e6():
    with pytest.raises(wave1d.Wave1DError):
        wave1d.Nufft(np.zeros(4), 8, 1e-8, 1)


def test_nufft_batched_instances():
    """wave1d_nufft_plan_many: five instances of different sizes and layouts (1 point, a cluster,
    points on the periodic seam, uniform, a ragged 37) in one plan, K = 300; each instance's
    type-1 and type-2 against its own direct sums, FP64 and mixed."""
    rng = np.random.default_rng(5)
    K = 300
    sets = [np.array([0.3]),
            -1.0 + 0.01 * rng.standard_normal(2500),
            np.concatenate([np.pi - 1e-3 * rng.uniform(size=400), -np.pi + 1e-3 * rng.uniform(size=400)]),
            rng.uniform(-np.pi, np.pi, 3000),
            rng.uniform(-np.pi, np.pi, 37)]
    cs = [rng.uniform(0.5, 1.5, v.size) * np.where(rng.uniform(size=v.size) < 0.8, 1.0, -1.0) for v in sets]
    alphas = []
    for _ in sets:
        a = (rng.standard_normal(K + 1) + 1j * rng.standard_normal(K + 1)) / (1.0 + np.arange(K + 1) / 50.0)
        a[0] = a[0].real
        alphas.append(a)
    import torch
    for precision, tol, bar in ((0, 1e-12, 1e-10), (1, 1e-6, 1e-6)):
        nu = wave1d.Nufft(sets, K, tol, precision)
        try:
            off = nu.offsets
            c_all = np.concatenate(cs)
            cd = torch.tensor(c_all[nu.perm], dtype=torch.float64, device="cuda")
            Sd = torch.zeros(len(sets) * 2 * (K + 1), dtype=torch.float64, device="cuda")
            ad = torch.tensor(np.concatenate([np.stack([a.real, a.imag], 1).reshape(-1) for a in alphas]),
                              dtype=torch.float64, device="cuda")
            ud = torch.zeros(nu.M, dtype=torch.float64, device="cuda")
            nu.type1(cd, Sd)
            nu.type2(ad, ud)
            torch.cuda.synchronize()
            S = Sd.cpu().numpy().reshape(len(sets), K + 1, 2)
            u = np.empty(nu.M)
            u[nu.perm] = ud.cpu().numpy()
        finally:
            nu.close()
        for i, (x, c, a) in enumerate(zip(sets, cs, alphas)):
            eS = _rel(S[i, :, 0] + 1j * S[i, :, 1], wfp.type1(c, x, K))
            eu = _rel(u[off[i]:off[i + 1]], wfp.type2(a, x))
            print(f"batched precision {precision} instance {i} (M={x.size}): type-1 {eS:.2e} type-2 {eu:.2e}")
            assert eS < bar and eu < bar


@pytest.mark.parametrize("precision,tol,bar_pass,bar_full", [(0, 1e-12, 1e-13, 1e-10), (1, 1e-6, 2e-6, 2e-6)])
def test_nufft_adjoint_identities(precision, tol, bar_pass, bar_full):
    """Interpolation is the transpose of spreading (same kernel values): <spread c, g> = <c, interp g>
    for any c, g.  And for real c, sum_j c_j u_j with u = type-2(alpha) equals
    2 pi (alpha_0 S_0 + 2 Re sum_{k>=1} alpha_k conj(S_k)) with S = type-1(c) (both transforms
    approximate exact adjoints to the tolerance).  Clustered points with a dense cell, M = 4000."""
    import torch
    rng = np.random.default_rng(17)
    x = np.concatenate([0.7 + 1e-3 * rng.standard_normal(1500), rng.uniform(-np.pi, np.pi, 2500)])
    K = 500
    nu = wave1d.Nufft(x, K, tol, precision)
    try:
        c = torch.tensor(rng.standard_normal(x.size), dtype=torch.float64, device="cuda")
        g = torch.tensor(rng.standard_normal(nu.nf), dtype=torch.float64, device="cuda")
        sc = torch.zeros(nu.nf, dtype=torch.float64, device="cuda")
        ig = torch.zeros(x.size, dtype=torch.float64, device="cuda")
        nu.spread(c, sc)
        nu.interp(g, ig)
        lhs, rhs = float(torch.dot(sc, g)), float(torch.dot(c, ig))
        scale = float(torch.linalg.norm(sc) * torch.linalg.norm(g))
        e_pass = abs(lhs - rhs) / scale
        alpha = (rng.standard_normal(K + 1) + 1j * rng.standard_normal(K + 1)) / (1.0 + np.arange(K + 1) / 100.0)
        alpha[0] = alpha[0].real
        ad = torch.tensor(np.stack([alpha.real, alpha.imag], 1).reshape(-1), dtype=torch.float64, device="cuda")
        S = torch.zeros(2 * (K + 1), dtype=torch.float64, device="cuda")
        u = torch.zeros(x.size, dtype=torch.float64, device="cuda")
        nu.type1(c, S)
        nu.type2(ad, u)
        torch.cuda.synchronize()
        Sh = S.cpu().numpy()
        Sc = Sh[0::2] + 1j * Sh[1::2]
        lhs2 = float(torch.dot(c, u))
        rhs2 = 2 * np.pi * float(np.real(alpha[0] * Sc[0] + 2 * np.sum(alpha[1:] * np.conj(Sc[1:]))))
        scale2 = float(torch.linalg.norm(c) * torch.linalg.norm(u))
        e_full = abs(lhs2 - rhs2) / scale2
    finally:
        nu.close()
    print(f"adjoint precision {precision}: spread/interp {e_pass:.2e}, type-1/type-2 {e_full:.2e}")
    assert e_pass < bar_pass and e_full < bar_full



@pytest.mark.parametrize("precision,tol", [(1, 1e-6), (0, 1e-12)])
def test_autotuned_spreading_matches_the_default_split(precision, tol):
    """The autotuner keeps one of its candidate splits; the spread it gives equals the default
    split's to rounding, and type-1 through it still matches the direct sums."""
    import torch
    from paper_2507_07823_gb300 import workloads as W
    ws = W.config3_instances(n_instances=16, m_range=(1e2, 3e3))
    nu = wave1d.Nufft([w.x for w in ws], 3141, tol, precision=precision)
    try:
        rng = np.random.default_rng(4)
        c = torch.from_numpy(rng.standard_normal(nu.M)).cuda()
        g0 = torch.zeros(nu.B * nu.nf, dtype=torch.float64, device="cuda")
        g1 = torch.zeros_like(g0)
        nu.spread(c, g0)
        cells, points = nu.autotune(c, g1, reps=3)
        nu.spread(c, g1)
        assert cells > 0 and points > 0
        assert float(torch.max(torch.abs(g1 - g0))) <= 1e-6 * float(torch.max(torch.abs(g0)))
    finally:
        nu.close()
