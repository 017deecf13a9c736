"""GPU parity of the differentiable loss L = sum_o (rho_k - rho_t)^2 and of its
hand-written backward kernels: against the FP64 oracle's forward, its
analytic gradients, and FP64 central finite differences (step 1e-3)."""
import numpy as np
import pytest

import oracle as O
from oracle import diff as D
from paper_2502_01286_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sncc():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    from paper_2502_01286_gb300 import build
    build.build()
    from paper_2502_01286_gb300 import sncc as mod
    return mod


@pytest.fixture(scope="module")
def problem(sncc):
    """512 x 512 float source, 48 x 48 template, fixed segmentation at std
    threshold 12 (computed on the template rounded to uint8); segment values
    start at the float means and are perturbed so the loss is not at a
    stationary point."""
    f, t, org, sigma = synth.case_diff()
    seg = sncc.build_segments(np.rint(np.clip(t, 0, 255)).astype(np.uint8), sigma)
    rects = seg.table
    k0 = np.array([t[y:y + h, x:x + w].mean() for x, y, w, h in rects], np.float64)
    k0 = k0 + np.random.default_rng(1).normal(0.0, 1.5, size=len(k0))
    return f, t, rects, k0


def rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-30))


def test_diff_forward_vs_oracle(sncc, problem):
    f, t, rects, k0 = problem
    N, M = f.shape
    pb = sncc.DiffProblem(t, rects, M, N)
    fd = torch.as_tensor(f).cuda()
    kd = torch.as_tensor(k0.astype(np.float32)).cuda()
    rho_k, rho_t, loss = sncc._diff_forward(pb, fd, kd)
    torch.cuda.synchronize()
    ref = D.forward(f.astype(np.float64), t.astype(np.float64), rects, k0.astype(np.float32).astype(np.float64))
    assert np.abs(rho_k.cpu().numpy() - ref["rho_k"]).max() <= 1e-5
    assert np.abs(rho_t.cpu().numpy() - ref["rho_t"]).max() <= 1e-5
    assert abs(float(loss.item()) - ref["loss"]) <= 1e-5 * ref["loss"]


def test_diff_backward_vs_oracle_and_finite_differences(sncc, problem):
    f, t, rects, k0 = problem
    N, M = f.shape
    k32 = k0.astype(np.float32)
    pb = sncc.DiffProblem(t, rects, M, N)
    fd = torch.as_tensor(f).cuda().requires_grad_(True)
    kd = torch.as_tensor(k32).cuda().requires_grad_(True)
    loss = pb.loss(fd, kd)
    loss.backward()
    torch.cuda.synchronize()
    gk = kd.grad.cpu().numpy()
    gf = fd.grad.cpu().numpy()
    f64, t64, k64 = f.astype(np.float64), t.astype(np.float64), k32.astype(np.float64)
    ref = D.gradients(f64, t64, rects, k64)
    assert rel(gk, ref["dk"]) <= 1e-4
    assert rel(gf, ref["df"]) <= 1e-4
    # FP64 central differences of the loss, step 1e-3
    h = 1e-3
    rng = np.random.default_rng(7)
    js = rng.choice(len(k64), size=4, replace=False).tolist() + [int(np.abs(ref["dk"]).argmax())]
    for j in js:
        kp, km = k64.copy(), k64.copy()
        kp[j] += h
        km[j] -= h
        num = (D.forward(f64, t64, rects, kp)["loss"] - D.forward(f64, t64, rects, km)["loss"]) / (2 * h)
        assert abs(gk[j] - num) <= 1e-4 * np.abs(ref["dk"]).max(), (j, gk[j], num)
    ys, xs = np.unravel_index(np.argsort(-np.abs(ref["df"]).ravel())[:3], f.shape)
    for y, x in list(zip(ys.tolist(), xs.tolist())) + [(5, 5), (300, 200)]:
        fp, fm = f64.copy(), f64.copy()
        fp[y, x] += h
        fm[y, x] -= h
        num = (D.forward(fp, t64, rects, k64)["loss"] - D.forward(fm, t64, rects, k64)["loss"]) / (2 * h)
        assert abs(gf[y, x] - num) <= 1e-4 * np.abs(ref["df"]).max(), (y, x, gf[y, x], num)


def test_refit_segment_values_reduces_loss(sncc, problem):
    """Gradient steps on the segment values at a fixed segmentation make
    segmented NCC track exact NCC more closely."""
    f, t, rects, k0 = problem
    N, M = f.shape
    pb = sncc.DiffProblem(t, rects, M, N)
    fd = torch.as_tensor(f).cuda()
    k, losses = sncc.refit_segment_values(pb, fd, k0, steps=40, lr=0.5)
    assert losses[-1] < 0.7 * losses[0]
    ref0 = D.forward(f.astype(np.float64), t.astype(np.float64), rects, k0)["loss"]
    ref1 = D.forward(f.astype(np.float64), t.astype(np.float64), rects, k.cpu().numpy().astype(np.float64))["loss"]
    assert ref1 < ref0


def test_backward_after_another_forward_on_the_same_workspace(sncc, problem):
    """Two losses on one DiffProblem, then backward of the first: the
    workspace holds the second forward, so the first backward must redo its
    own forward and give the same gradients as a clean forward + backward."""
    f, t, rects, k0 = problem
    N, M = f.shape
    pb = sncc.DiffProblem(t, rects, M, N)
    k32 = k0.astype(np.float32)
    fa = torch.as_tensor(f).cuda().requires_grad_(True)
    ka = torch.as_tensor(k32).cuda().requires_grad_(True)
    fb = torch.as_tensor(np.ascontiguousarray(f[::-1])).cuda().requires_grad_(True)
    kb = torch.as_tensor(k32[::-1].copy()).cuda().requires_grad_(True)
    la = pb.loss(fa, ka)
    lb = pb.loss(fb, kb)
    la.backward()
    lb.backward()
    fc = torch.as_tensor(f).cuda().requires_grad_(True)
    kc = torch.as_tensor(k32).cuda().requires_grad_(True)
    pb.loss(fc, kc).backward()
    fd2 = torch.as_tensor(np.ascontiguousarray(f[::-1])).cuda().requires_grad_(True)
    kd2 = torch.as_tensor(k32[::-1].copy()).cuda().requires_grad_(True)
    pb.loss(fd2, kd2).backward()
    torch.cuda.synchronize()
    # dL/df has no cross-block reduction and repeats bit for bit; dL/dk sums
    # block partials with atomics, so it repeats to rounding
    assert torch.equal(fa.grad, fc.grad) and torch.equal(fb.grad, fd2.grad)
    for g1, g2 in ((ka.grad, kc.grad), (kb.grad, kd2.grad)):
        assert float((g1 - g2).abs().max()) <= 1e-6 * float(g2.abs().max())
    assert float((ka.grad - kb.grad).abs().max()) > 1e-3 * float(kb.grad.abs().max())


def test_diff_multi_block_template_vs_oracle(sncc):
    """A 150 x 100 template (blocks of 64 x 64: three columns of blocks, the
    last 22 wide, and two rows, the last 36 high) on a 200 x 150 float
    source: the loss, both maps and both gradients against the FP64 oracle,
    and one segment value and two source pixels against FP64 central
    differences (step 1e-3)."""
    f, t, org, sigma = synth.case_diff(M=200, N=150, W=150, H=100)
    seg = sncc.build_segments(np.rint(np.clip(t, 0, 255)).astype(np.uint8), sigma)
    rects = seg.table
    k0 = np.array([t[y:y + h, x:x + w].mean() for x, y, w, h in rects], np.float64)
    k0 = k0 + np.random.default_rng(2).normal(0.0, 1.5, size=len(k0))
    k32 = k0.astype(np.float32)
    N, M = f.shape
    pb = sncc.DiffProblem(t, rects, M, N)
    fd = torch.as_tensor(f).cuda().requires_grad_(True)
    kd = torch.as_tensor(k32).cuda().requires_grad_(True)
    rho_k, rho_t, loss0 = sncc._diff_forward(pb, fd.detach(), kd.detach())
    torch.cuda.synchronize()
    f64, t64, k64 = f.astype(np.float64), t.astype(np.float64), k32.astype(np.float64)
    ref = D.gradients(f64, t64, rects, k64)
    fw = D.forward(f64, t64, rects, k64)
    assert np.abs(rho_k.cpu().numpy() - fw["rho_k"]).max() <= 1e-5
    assert np.abs(rho_t.cpu().numpy() - fw["rho_t"]).max() <= 1e-5
    assert abs(float(loss0.item()) - fw["loss"]) <= 1e-5 * fw["loss"]
    loss = pb.loss(fd, kd)
    loss.backward()
    torch.cuda.synchronize()
    gk = kd.grad.cpu().numpy()
    gf = fd.grad.cpu().numpy()
    assert rel(gk, ref["dk"]) <= 1e-4
    assert rel(gf, ref["df"]) <= 1e-4
    h = 1e-3
    j = int(np.abs(ref["dk"]).argmax())
    kp, km = k64.copy(), k64.copy()
    kp[j] += h
    km[j] -= h
    num = (D.forward(f64, t64, rects, kp)["loss"] - D.forward(f64, t64, rects, km)["loss"]) / (2 * h)
    assert abs(gk[j] - num) <= 1e-4 * np.abs(ref["dk"]).max(), (j, gk[j], num)
    y, x = np.unravel_index(int(np.abs(ref["df"]).argmax()), f.shape)
    for (py, px) in [(int(y), int(x)), (120, 70)]:
        fp, fm = f64.copy(), f64.copy()
        fp[py, px] += h
        fm[py, px] -= h
        num = (D.forward(fp, t64, rects, k64)["loss"] - D.forward(fm, t64, rects, k64)["loss"]) / (2 * h)
        assert abs(gf[py, px] - num) <= 1e-4 * np.abs(ref["df"]).max(), (py, px, gf[py, px], num)


def _random_diff_problems(n=4, seed=2026120303):
    """Seeded random problems: templates of 4 to 130 pixels a side (one block
    or several 64 x 64 blocks), sources 8 to 120 columns and rows larger, std
    thresholds 6 to 16."""
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        W, H = int(g.integers(4, 131)), int(g.integers(4, 131))
        M, N = W + int(g.integers(8, 120)), H + int(g.integers(8, 100))
        out.append((i, M, N, W, H, float(g.choice([6.0, 9.0, 12.0, 16.0])), int(g.integers(0, 1 << 30))))
    return out


@pytest.mark.parametrize("i,M,N,W,H,sigma,seed", _random_diff_problems())
def test_diff_random_problems_vs_oracle(sncc, i, M, N, W, H, sigma, seed):
    """Both maps and the loss within 1e-5, both gradients within 1e-4
    relative of the FP64 oracle's analytic ones."""
    f, t, org, _ = synth.case_diff(M=M, N=N, W=W, H=H, seed=seed)
    seg = sncc.build_segments(np.rint(np.clip(t, 0, 255)).astype(np.uint8), sigma)
    rects = seg.table
    k0 = np.array([t[y:y + h, x:x + w].mean() for x, y, w, h in rects], np.float64)
    k0 = k0 + np.random.default_rng(seed).normal(0.0, 1.5, size=len(k0))
    k32 = k0.astype(np.float32)
    pb = sncc.DiffProblem(t, rects, M, N)
    fd = torch.as_tensor(f).cuda().requires_grad_(True)
    kd = torch.as_tensor(k32).cuda().requires_grad_(True)
    rho_k, rho_t, loss0 = sncc._diff_forward(pb, fd.detach(), kd.detach())
    loss = pb.loss(fd, kd)
    loss.backward()
    torch.cuda.synchronize()
    f64, t64, k64 = f.astype(np.float64), t.astype(np.float64), k32.astype(np.float64)
    fw = D.forward(f64, t64, rects, k64)
    ref = D.gradients(f64, t64, rects, k64)
    assert np.abs(rho_k.cpu().numpy() - fw["rho_k"]).max() <= 1e-5
    assert np.abs(rho_t.cpu().numpy() - fw["rho_t"]).max() <= 1e-5
    assert abs(float(loss0.item()) - fw["loss"]) <= 1e-5 * fw["loss"]
    assert abs(float(loss.item()) - fw["loss"]) <= 1e-5 * fw["loss"]
    assert rel(kd.grad.cpu().numpy(), ref["dk"]) <= 1e-4
    assert rel(fd.grad.cpu().numpy(), ref["df"]) <= 1e-4
