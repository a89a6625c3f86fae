"""The learned preconditioner on the GPU: the tcgen05 BF16 GEMM, the Fourier neural
operator's forward and backward passes against the FP64 oracle (oracle/fno.py), training,
and flexible GMRES (through the C ABI).

Tolerances.  The GEMM rounds its operands to BF16 (relative 2^-9) and accumulates in FP32:
against an FP64 product of the same BF16-rounded operands every entry is within
1e-4 * sum_k |a_mk| |b_nk| (FP32 accumulation of up to 16384 terms).  The network chains
about 30 such products per pass, each rounding its inputs to BF16, so its output and
gradients are compared with the FP64 oracle in the relative 2-norm at 3e-2 (forward) and
6e-2 (every gradient tensor).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dense, fno as ofno, gmres  # noqa: E402
from paper_1104_4263_gb300 import die, workloads as W  # noqa: E402


def _bf(t):
    return t.to(torch.bfloat16).to(torch.float64)


@pytest.mark.parametrize("M,N,K,batch,transpose_a", [(128, 64, 64, 1, False), (200, 70, 100, 1, False),
                                                     (300, 130, 333, 2, True), (32, 32, 4096, 3, False),
                                                     (5, 200, 17, 1, True)])
def test_gemm_bf16_matches_reference(M, N, K, batch, transpose_a):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(batch, K, M, generator=g).transpose(1, 2) if transpose_a else torch.randn(batch, M, K, generator=g)
    B = torch.randn(batch, N, K, generator=g)
    C0 = torch.randn(batch, M, N, generator=g)
    Ad, Bd, Cd = A.cuda(), B.cuda(), C0.clone().cuda()
    for beta in (0.0, 1.0):
        Cd.copy_(C0.cuda())
        out = die.gemm_bf16(Ad, Bd, Cd, alpha=0.5, beta=beta).cpu().double()
        ref = 0.5 * torch.bmm(_bf(A), _bf(B).transpose(1, 2)) + beta * C0.double()
        bound = 0.5 * torch.bmm(_bf(A).abs(), _bf(B).abs().transpose(1, 2))
        assert torch.all((out - ref).abs() <= 1e-4 * bound + 1e-6), float((out - ref).abs().max())


def _flat_params(p, L):
    parts = [p["P"], p["p"]]
    for l in range(L):
        parts += [p[f"W{l}"], p[f"w{l}"]]
        for nm in (f"R1_{l}", f"R2_{l}"):
            parts.append(np.stack([p[nm].real, p[nm].imag], axis=-1))
    parts += [p["Q1"], p["q1"], p["Q2"], p["q2"]]
    return np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in parts])


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_fno_forward_backward_match_oracle():
    """Same parameters and inputs on both sides (a 32 x 32 grid, 6 modes, width 8, two
    layers, batch 2): output, every parameter gradient and the input gradient."""
    c_in, c_out, width, m, L, hid, H, Wd, B = 3, 2, 8, 6, 2, 16, 32, 32, 2
    rng = np.random.default_rng(7)
    p = ofno.init_params(rng, c_in, c_out, width, m, L, hid)
    net = die.FNO(c_in, c_out, width, m, L, hid, H, Wd, max_batch=B)
    flat = _flat_params(p, L)
    assert flat.size == net.n_params
    net.set_params(flat)
    x = rng.standard_normal((B, c_in, H, Wd))
    gy = rng.standard_normal((B, c_out, H, Wd))
    y = net.forward(torch.from_numpy(x).float().cuda()).cpu().numpy()
    ref, tapes, grads = [], [], None
    for b in range(B):
        yb, tape = ofno.forward(p, x[b])
        ref.append(yb)
        gb = ofno.backward(p, tape, gy[b])
        grads = gb if grads is None else {k: grads[k] + gb[k] for k in grads if k != "x"} | {"x": None}
        tapes.append(gb["x"])
    assert _rel(y, np.stack(ref)) < 3e-2
    net.zero_grads()
    gx = net.backward(torch.from_numpy(gy).float().cuda(), want_gx=True).cpu().numpy()
    assert _rel(gx, np.stack(tapes)) < 6e-2
    g_gpu = net.get_grads()
    g_ref = _flat_params({k: v for k, v in grads.items() if k != "x"} | {"layers": L}, L)
    # tensor by tensor
    off = 0
    names = ["P", "p"] + [f"{n}{l}" for l in range(L) for n in ("W", "w", "R1_", "R2_")] + ["Q1", "q1", "Q2", "q2"]
    for nm in names:
        a = grads[nm]
        size = a.size * (2 if np.iscomplexobj(a) else 1)
        e = _rel(g_gpu[off:off + size], g_ref[off:off + size])
        assert e < 6e-2, (nm, e)
        off += size
    assert off == g_gpu.size


def test_fno_training_reduces_loss():
    """A few hundred Adam steps on a fixed synthetic regression (the target is a smooth
    linear map of the input) cut the loss by an order of magnitude."""
    c_in, c_out, H, Wd, B = 2, 1, 32, 32, 8
    net = die.FNO(c_in, c_out, 16, 6, 2, 32, H, Wd, max_batch=B)
    rng = np.random.default_rng(3)
    p = ofno.init_params(rng, c_in, c_out, 16, 6, 2, 32)
    net.set_params(_flat_params(p, 2) * 0.5)
    x = rng.standard_normal((B, c_in, H, Wd))
    kx = np.fft.fftfreq(Wd)[None, :]
    ky = np.fft.fftfreq(H)[:, None]
    filt = np.exp(-40 * (kx ** 2 + ky ** 2))
    t = np.real(np.fft.ifft2(np.fft.fft2(x[:, 0] - 0.5 * x[:, 1]) * filt))[:, None]
    xt, tt = torch.from_numpy(x).float().cuda(), torch.from_numpy(t).float().cuda()
    losses = [net.train_step(xt, tt, 2e-3) for _ in range(300)]
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])


def test_fgmres_identity_preconditioner_is_gmres():
    """With no network (the identity preconditioner) flexible GMRES is GMRES: on the 32^2
    cylinder its first cycle is the oracle's flexible GMRES cycle (same Krylov space: the
    same iterate to rounding), and both reach the same solution (the step counts of many
    restarted cycles drift apart by rounding, as for the restarted solver)."""
    p = W.config1(32)
    op = die.Operator(p.eps_r, p.h)
    b = op.plane_wave(0.0)
    A = dense.dense_A(p.eps_r, p.h)
    mv = lambda v: dense.matvec(A, v)
    x1, r1 = die.fgmres(op, b, restart=20, tol=1e-14, max_iters=20, reorth_eta=1.0)
    ref1 = gmres.fgmres(mv, b.cpu().numpy(), 20, 1e-14, 20)
    assert r1["iters"] == ref1.iters == 20
    assert _rel(x1.cpu().numpy(), ref1.x) < 1e-10
    x, rep = die.fgmres(op, b, restart=20, tol=1e-10, max_iters=4000, reorth_eta=1.0)
    ref = gmres.fgmres(mv, b.cpu().numpy(), 20, 1e-10, 4000)
    assert rep["converged"] and ref.converged
    assert abs(rep["iters"] - ref.iters) <= 0.1 * ref.iters, (rep["iters"], ref.iters)
    assert _rel(x.cpu().numpy(), ref.x) < 1e-7


def test_fgmres_with_untrained_network_converges():
    """A network with zero weights is the identity map M(v) = v; a randomly initialised one
    is a nonlinear step-dependent preconditioner: flexible GMRES still reaches the direct
    solution, and the fallback (regularised, deflated GMRES) finishes a solve the flexible
    iteration leaves unconverged."""
    n = 32
    p = W.config1(n)
    op = die.Operator(p.eps_r, p.h)
    b = op.plane_wave(0.3)
    A = dense.dense_A(p.eps_r, p.h)
    xd = np.linalg.solve(A, b.cpu().numpy().reshape(-1))
    net = die.FNO(6, 4, 8, 6, 2, 16, n, n, max_batch=1)
    z = net.precondition(op, b)
    assert torch.equal(z, b)          # zero weights: M(v) = v
    rng = np.random.default_rng(11)
    net.set_params(0.05 * _flat_params(ofno.init_params(rng, 6, 4, 8, 6, 2, 16), 2))
    x, rep = die.fgmres(op, b, net=net, restart=20, tol=1e-8, max_iters=3000)
    assert rep["converged"] and not rep["used_fallback"]
    assert _rel(x.cpu().numpy().reshape(-1), xd) < 1e-5
    # the fallback: regularised FP32-inner GMRES(60) (no deflation: this rotationally symmetric
    # object has degenerate eigenvalue pairs that a small rank can split; GMRES(20) on the
    # regularised system stagnates for this incidence angle)
    x2, rep2 = die.fgmres(op, b, net=net, restart=10, tol=1e-6, max_iters=5,
                          fallback_restart=60, fallback_iters=5000)
    assert rep2["used_fallback"] and rep2["converged"] and rep2["rel_res_orig"] <= 1e-6, rep2
    assert _rel(x2.cpu().numpy().reshape(-1), xd) < 1e-3


def test_learned_preconditioner_trains_and_helps():
    """The whole learned pipeline at 64^2 (h = 1/60): 384 solver-generated pairs (every 32nd
    from a regularised GMRES solve of a plane wave, the rest from one product), training on
    the GPU, then a held-out field solved without the network (regularised + deflated
    GMRES(100)) and with it (flexible GMRES(30), then the former).  The trained network must
    fit its training pairs better than the identity map it starts as, and both solves must
    reach 1e-5 on ||b - A u|| / ||b||.  What the network gains (iterations, seconds, the
    residual of its initial guess) is printed; at this training budget (144 Adam steps) it
    gains nothing, and the bench measures it at 128^2 with 20000 pairs."""
    from paper_1104_4263_gb300 import learned
    data = learned.make_dataset(384, n=64, solve_every=32)
    net = learned.default_network(64, max_batch=16)
    e0 = learned.relative_error(net, data)
    losses, _ = learned.train(net, data, epochs=6)
    e1 = learned.relative_error(net, data)
    assert abs(e0 - 1.0) < 1e-6 and e1 < 0.9 * e0, (e0, e1, losses)
    rows = learned.evaluate(net, 1, n=64, tol=1e-5, r_defl=6, max_iters=10000, first=learned.HELD_OUT_BASE + 1)
    for r in rows:
        assert r["without_network"]["converged"] and r["with_network"]["converged"], r
        assert math.isfinite(r["initial_guess_rel_res"]), r
    print("learned 64^2:", [(r["without_network"]["iters"], r["with_network"]["iters"],
                             round(r["initial_guess_rel_res"], 3)) for r in rows])
