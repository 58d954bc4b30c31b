"""What the trained spectral neural operator gains as the coarse propagator of Parareal (its use in
the surrogate-accelerated solve), against two coarse propagators without learning: the identity (the
operator with a zero projection, u_hat = u) and one ETDRK2 step of the window's length (50 tau here:
the exponential integrator's own large step). The fine propagator is the plain batched ETDRK2
solver. For each, with rejected windows falling back to the plain solver (threshold 1e-2): the
Parareal iterations and fallbacks to reach the plain solver's final state to rel L2 <= 1e-3, and the
wall time against the plain batched solve; without fallbacks: the correction of every iteration.

The serial length of a run, in windows of the fine solver, is its iterations (each one batched fine
sweep over all windows) plus its fallbacks (each one window advanced alone); the plain solve is
`windows` of them. A smaller operator than the full workload keeps training short (N = 64, C = 16,
M = 12, L = 2; 400 trajectories; windows of 10 steps). Asserted: every propagator reaches the
tolerance with and without fallbacks; the trained operator's first correction is smaller than the
identity's and its serial length is no longer (the gain of learning); the ETDRK2 step, exact for the
linear part, is no longer than the identity either."""
import time

import numpy as np
import pytest

from paper_2209_11922_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = inputs.SnoWorkload("gain", N=64, C=16, M=12, L=2, window=10, tau=1e-2, trajectories=400, traj_steps=40,
                       batch=16, windows=4)


def test_trained_operator_gain_over_nonlearned_coarse_propagators():
    from paper_2209_11922_gb300.etd import Batch
    from paper_2209_11922_gb300.sno import Parareal, Sno
    from paper_2209_11922_gb300.sno_train import make_pairs, train

    B, Wn = W.batch, W.windows
    u_in, u_out, Dtr = make_pairs(W, range(W.trajectories))
    sno = Sno(W.N, W.C, W.M, W.L, B)
    sno.set_params(W.init_weights())
    hist = train(sno, u_in, u_out, Dtr, 8, B, lr=3e-3, seed=W.seed)
    print(f"training loss: first epoch {hist[0]:.3e}, last {hist[-1]:.3e}")
    assert hist[-1] < hist[0]
    ident = Sno(W.N, W.C, W.M, W.L, B)
    P0 = W.init_weights()
    P0["Wq"] = np.zeros_like(P0["Wq"])      # zero projection: u_hat = u exactly
    ident.set_params(P0)

    tid = [10 ** 6 + b for b in range(B)]
    D = [W.D(i) for i in tid]
    u0 = torch.from_numpy(np.stack([W.u0(i) for i in tid]).astype(np.float32)).cuda()
    ref = u0.clone()
    with Batch([(W.N, W.N)] * B, D, W.tau, 2, "f32") as plain:
        plain.run([ref[b] for b in range(B)], Wn * W.window)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            w = u0.clone()
            plain.run([w[b] for b in range(B)], Wn * W.window)
        torch.cuda.synchronize()
        t_plain = (time.perf_counter() - t0) / 5

    def err_of(out):
        return max(float((torch.linalg.vector_norm(out[b] - ref[b]) / torch.linalg.vector_norm(ref[b])).item())
                   for b in range(B))

    results = {}
    for name, coarse in (("trained SNO", sno), ("identity", ident), ("ETDRK2 step of 10 tau", None)):
        pr = Parareal(coarse, W.N, D, W.tau, W.window, Wn)
        out, st = pr.run(u0, Wn, 1e-5, 1e-2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            out, st = pr.run(u0, Wn, 1e-5, 1e-2)
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) / 3
        r = dict(st, err=err_of(out), time_vs_plain=t / t_plain, serial=st["iterations"] + st["fallbacks"])
        out, st = pr.run(u0, Wn, 1e-5, 1e30)
        r.update(err_nofb=err_of(out), corrections_nofb=st["correction"])
        results[name] = r
        pr.close()
    for name, r in results.items():
        print(f"{name}: iterations {r['iterations']}, fallbacks {r['fallbacks']}, serial windows {r['serial']} of "
              f"{Wn}, final rel L2 {r['err']:.2e}, first correction {r['correction'][0]:.3e}, time / plain solve "
              f"{r['time_vs_plain']:.2f}; without fallbacks: corrections "
              f"{' '.join(f'{c:.2e}' for c in r['corrections_nofb'])}, final rel L2 {r['err_nofb']:.2e}")
    for r in results.values():
        assert r["err"] <= 1e-3 and r["err_nofb"] <= 1e-3
    s, i, e = results["trained SNO"], results["identity"], results["ETDRK2 step of 10 tau"]
    assert s["correction"][0] < i["correction"][0]
    assert s["serial"] <= i["serial"]
    assert e["serial"] <= i["serial"]
    sno.close()
    ident.close()
