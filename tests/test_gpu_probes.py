"""Device Voigt and E_n, called through the C ABI probes (same device code as
the kernels), against the FP64 oracle at the same (FP32-rounded) inputs."""
import numpy as np
import pytest

import paper_2607_24141_gb300 as pz

pytestmark = pytest.mark.gpu


def voigt_gpu(a, v):
    import torch
    at = torch.tensor(a, dtype=torch.float32, device="cuda")
    vt = torch.tensor(v, dtype=torch.float32, device="cuda")
    H = torch.empty_like(at)
    dH = torch.empty_like(at)
    pz.pz_probe_voigt(at, vt, H, dH)
    torch.cuda.synchronize()
    return H.cpu().numpy().astype(np.float64), dH.cpu().numpy().astype(np.float64)


def test_fp32_voigt_accuracy(oracle):
    a = np.logspace(-4, 1.5, 90).astype(np.float32)
    v = np.concatenate([np.linspace(0, 8, 321), np.linspace(8, 30, 177),
                        np.logspace(np.log10(30), np.log10(2500), 80)]).astype(np.float32)
    A, V = np.meshgrid(a, v, indexing="ij")
    A, V = A.ravel(), V.ravel()
    H, dH = voigt_gpu(A, V)
    Hr, _, dHr = oracle.voigt(A.astype(np.float64), V.astype(np.float64))
    x2 = V.astype(np.float64) ** 2
    # the Gaussian core's condition number w.r.t. an FP32 input is ~2 v^2
    bound = 2e-6 + 2 * x2 * 6e-8 * np.exp(-x2) / Hr
    err = np.abs(H / Hr - 1)
    assert np.all(err < bound), (float(err.max()), A[np.argmax(err / bound)], V[np.argmax(err / bound)])
    # dH/da: relative to the local scale |dH/da| + H/max(a, 1)
    scale = np.abs(dHr) + Hr / np.maximum(A, 1.0)
    derr = np.abs(dH - dHr) / scale
    assert derr.max() < 3e-5, (float(derr.max()), A[np.argmax(derr)], V[np.argmax(derr)])


def test_fp64_expn(oracle):
    import torch
    edges = np.array([2.0 ** -40, 2.0, 40.0, 0.5, 1.0, 0.25])
    x = np.concatenate([[0.0], np.logspace(-16, -11, 40), np.logspace(-12, 0, 200), np.linspace(1, 3, 200),
                        np.linspace(3, 745, 400), np.linspace(38.0, 42.0, 64),
                        edges * (1 - 1e-15), edges, edges * (1 + 1e-15),
                        np.random.default_rng(3).uniform(0.0, 50.0, 500)])
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    out = torch.empty(5 * x.size, dtype=torch.float64, device="cuda")
    pz.pz_probe_expn(xt, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(5, -1)
    for k, n in enumerate((2, 3, 4)):
        ref = oracle.expn(n, x)
        m = ref > 1e-290
        err = np.abs(got[k][m] / ref[m] - 1)
        small = m & (x < 2.0)
        print("E_%d: max rel err %.3g (x < 2: %.3g)" % (n, err.max(), np.max(np.abs(got[k][small] / ref[small] - 1))))
        assert err.max() < 5e-14, n
    # the scattering kernels' E_2, E_3 (from the E_3 table): the same bound up to x = 40,
    # zero beyond
    near = x <= 40.0
    for k, n in ((3, 2), (4, 3)):
        ref = oracle.expn(n, x)
        err = np.abs(got[k][near] / ref[near] - 1)
        print("scattering E_%d: max rel err %.3g" % (n, err.max()))
        assert err.max() < 5e-14, n
        assert np.all(got[k][~near] == 0.0)


def test_pipe_probes_are_plausible():
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    fma = pz.pz_probe_pipe(0, 2048)
    rcp = pz.pz_probe_pipe(1, 2048)
    # between a quarter of the lane-count rate at 1 GHz and the lane-count rate at 2.5 GHz
    assert 0.25 * n_sm * 128 * 1e9 < fma < n_sm * 256 * 2.5e9
    assert 0.25 * n_sm * 16 * 1e9 < rcp < n_sm * 64 * 2.5e9
    # FP64: at least one FMA per SM per 4 ns, and far below the FP32 rate on this part
    dfma = pz.pz_probe_pipe(2, 256)
    assert n_sm * 0.25e9 < dfma < fma / 4, (dfma, fma)
    print("pipe probes: FP32 %.3g /s, MUFU %.3g /s, FP64 FMA %.3g /s" % (fma, rcp, dfma))
    with pytest.raises(pz.PzError) as e:
        pz.pz_probe_pipe(3, 16)
    assert e.value.status == pz.PZ_EINVAL
