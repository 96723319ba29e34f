"""GPU learned preconditioner (through the C ABI) against the FP64 oracle.

Tolerances, derived from BF16's unit roundoff u = 2^-8 (8-bit significand, round to nearest).
Every stored activation is rounded to BF16; on the tensor-core path the transported
neighbour values and the weights are rounded to BF16 as MMA operands as well, while the
FP32 accumulation (at most 17 x 8 x 3 terms, 2^-24 each) is negligible against u.  A term of
an 8 -> 8 layer therefore carries k = 3 independent roundings on the tensor cores (operand,
weight, stored output) and k = 1 on the CUDA cores (stored output).  Modelling each rounding
as an independent relative error uniform in [-u, u] (variance u^2/3), a sum of many terms
whose magnitudes do not cancel beyond random phases has a norm-wise relative error of rms
u sqrt(k/3), and errors of successive linear layers add in quadrature.  For the network
1 -> 8 -> 8 -> 8 -> 1 (L = 4 layers, plus the rounding of the input):
    forward, tensor cores:  u sqrt((3L + 1)/3) = 2.08 u = 8.1e-3   (the 1 -> 8 and 8 -> 1
                            layers run on the CUDA cores; counting them as 3 is an upper bound)
    forward, CUDA cores:    u sqrt((L + 1)/3)  = 1.29 u = 5.0e-3
    weight gradient:        the activations of layer l (forward path) times the output
                            gradient carried back through the layers above it (each a forward
                            layer with conjugate weights) and the rounded loss gradient:
                            at most k = (3L + 1) + 3(L - 1) + 1 = 23 -> u sqrt(23/3) = 1.1e-2
The tests allow FOUR times these rms estimates norm-wise (forward, loss, every layer's
gradient), and five times per tap of the gradient (17 taps x C_out x C_in weights each) and
per 128-site block of the output.  A transposed or wrongly conjugated tap, a dropped
direction or a stale tile gives errors of order one relative to the quantity checked.
Flexible CG with the network must reach a true FP64 residual <= 1e-10 (recomputed by the
oracle).
"""
import os

import numpy as np
import pytest
import torch

import oracle
from hisq_inputs import fields

hisq = pytest.importorskip("paper_2306_01098_gb300.hisq")

pytestmark = pytest.mark.gpu

NTAP = 17
U_BF16 = 2.0 ** -8
L = 4
RMS_FWD_TC = U_BF16 * np.sqrt((3 * L + 1) / 3)
RMS_FWD_CC = U_BF16 * np.sqrt((L + 1) / 3)
RMS_GRAD = U_BF16 * np.sqrt(((3 * L + 1) + 3 * (L - 1) + 1) / 3)
TOL_FWD = {1: 4 * RMS_FWD_TC, 0: 4 * RMS_FWD_CC}
TOL_GRAD = 4 * RMS_GRAD
TOL_GRAD_TAP = 5 * RMS_GRAD


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rand_weights(chans, seed, scale=0.4):
    rng = np.random.default_rng(seed)
    ws = []
    for l in range(len(chans) - 1):
        n = NTAP * chans[l + 1] * chans[l]
        w = scale * (rng.normal(size=n) + 1j * rng.normal(size=n)) / np.sqrt(NTAP * chans[l])
        ws.append(w)
    return np.concatenate(ws)


def check_gradient(g, g_o, chans):
    """Norm-wise, per layer and per tap (the C_out x C_in weights of one transport)."""
    assert rel(g, g_o) <= TOL_GRAD
    off, worst = 0, 0.0
    for l in range(len(chans) - 1):
        n = chans[l + 1] * chans[l]
        gl, gol = g[off:off + NTAP * n], g_o[off:off + NTAP * n]
        assert rel(gl, gol) <= TOL_GRAD, l
        for tap in range(NTAP):
            e = rel(gl[tap * n:(tap + 1) * n], gol[tap * n:(tap + 1) * n])
            worst = max(worst, e)
            assert e <= TOL_GRAD_TAP, (l, tap, e)
        off += NTAP * n
    print(f"gradient: total {rel(g, g_o):.2e}, worst tap {worst:.2e} (tap tolerance {TOL_GRAD_TAP:.2e})")


@pytest.fixture(scope="module")
def small():
    dims = (6, 4, 4, 6)
    fat, lng = fields.recipe_links(dims, 0.5, 77)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16))
    return dims, ctx, fat.numpy(), lng.numpy()


@pytest.mark.parametrize("tensor_cores", [1, 0])
@pytest.mark.parametrize("link_prec", [hisq.F32, hisq.F16])
def test_network_forward_matches_oracle(small, link_prec, tensor_cores):
    tol = TOL_FWD[tensor_cores]
    dims, ctx, fat, lng = small
    net = hisq.Net(ctx, link_prec=link_prec, tensor_cores=tensor_cores)
    chans = [1, 8, 8, 8, 1]
    w = rand_weights(chans, 5)
    assert w.size == net.nw
    net.set_weights(w)
    b = fields.gaussian_source(dims, 300)[0]
    z = torch.empty_like(b).cuda()
    net.apply(b.cuda(), z)
    want = oracle.net_apply(dims, fat, lng, chans, w, b.numpy())
    assert rel(z.cpu().numpy(), want) <= tol


@pytest.mark.parametrize("dims", [(8, 8, 8, 10), (6, 6, 4, 10)])
def test_tensor_core_layers_match_cuda_core_layers(dims):
    # the 8 -> 8 layers' channel mixing on the tensor cores (BF16 operands, FP32 accumulation)
    # against the same network in FP32 on the CUDA cores: 128-site tiles, a ragged last tile
    # (V = 5120 = 40 tiles; V = 1440 = 11.25 tiles), identical weights, and the oracle
    fat, lng = fields.recipe_links(dims, 0.5, 79)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F32, hisq.F16))
    chans = [1, 8, 8, 8, 1]
    w = rand_weights(chans, 11)
    nets = [hisq.Net(ctx, tensor_cores=t) for t in (1, 0)]
    b = fields.gaussian_source(dims, 330)[0]
    outs = []
    for net in nets:
        net.set_weights(w)
        z = torch.empty_like(b).cuda()
        net.apply(b.cuda(), z)
        outs.append(z.cpu().numpy())
    want = oracle.net_apply(dims, fat.numpy(), lng.numpy(), chans, w, b.numpy())
    assert rel(outs[1], want) <= TOL_FWD[0]
    assert rel(outs[0], want) <= TOL_FWD[1]
    assert rel(outs[0], outs[1]) <= TOL_FWD[1]
    # every site was written: no site of the tensor-core output is left at zero
    assert np.abs(outs[0]).reshape(-1, 6).max(axis=1).min() > 0.0
    for net in nets:
        net.close()
    ctx.close()


def test_network_loss_and_gradient_match_oracle(small):
    dims, ctx, fat, lng = small
    net = hisq.Net(ctx)
    chans = [1, 8, 8, 8, 1]
    w = rand_weights(chans, 6)
    net.set_weights(w)
    b = fields.gaussian_source(dims, 301)[0]
    x = fields.gaussian_source(dims, 302)[0]
    loss, g = net.loss_grad(b.cuda(), x.cuda())
    loss_o, g_o = oracle.net_loss_grad(dims, fat, lng, chans, w, b.numpy(), x.numpy())
    assert abs(loss - loss_o) <= TOL_FWD[1] * loss_o
    check_gradient(g, g_o, chans)


def test_weights_roundtrip_and_save_load(small, tmp_path):
    dims, ctx, fat, lng = small
    net = hisq.Net(ctx, channels=4)
    w = rand_weights([1, 4, 4, 4, 1], 7)
    net.set_weights(w)
    assert np.abs(net.get_weights() - w).max() < 1e-6 * np.abs(w).max()
    p = str(tmp_path / "net.bin")
    net.save(p)
    net2 = hisq.Net.load(ctx, p)
    assert np.array_equal(net2.get_weights(), net.get_weights())


def test_training_lowers_loss_and_fcg_converges():
    dims, m = (8, 8, 8, 8), 0.05
    fat, lng = fields.recipe_links(dims, 0.5, 78)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16))
    npairs = 32
    B = fields.gaussian_source(dims, 310, npairs).cuda()
    X = torch.zeros_like(B)
    for k in range(0, npairs, 8):
        rc, st = ctx.cg(m, B[k:k + 8].contiguous(), X[k:k + 8], tol=1e-8, prec_sloppy=hisq.F32, prec_precise=hisq.F64)
        assert rc == hisq.OK
    X = X.contiguous()
    net = hisq.Net(ctx, epochs=4, batch=4, lr=3e-3)
    losses = net.train(B, X, 4)
    assert np.all(np.isfinite(losses)) and losses[-1] < losses[0]
    b = fields.gaussian_source(dims, 320)[0]
    x = torch.zeros_like(b).cuda()
    rc, st = hisq.fcg(ctx, m, b.cuda(), x, net=net, tol=1e-10, prec_precise=hisq.F64X)
    assert rc == hisq.OK
    r = b.numpy() - oracle.mdagm(dims, fat.numpy(), lng.numpy(), m, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b.numpy()) <= 1e-10
    # without a network flexible CG is CG
    x0 = torch.zeros_like(b).cuda()
    rc0, st0 = hisq.fcg(ctx, m, b.cuda(), x0, net=None, tol=1e-10, prec_precise=hisq.F64)
    xc = torch.zeros_like(b).cuda()
    rcc, stc = ctx.cg(m, b.cuda(), xc, tol=1e-10, prec_sloppy=hisq.F64)
    assert rc0 == hisq.OK and abs(st0.iterations - stc.iterations) <= 2
    print(f"losses {losses}, FCG(net) {st.iterations} iterations, FCG(1) {st0.iterations}, CG {stc.iterations}")
    # creation and training in one call (hisq_precond_train) give the same network up to the
    # order of the FP32 shared-memory accumulation of the weight gradient, which differs from
    # run to run; after these 32 Adam steps two trainings differ by about 1e-4 of the weights
    net1 = hisq.Net.trained(ctx, B, X, epochs=4, batch=4, lr=3e-3)
    w0, w1 = net.get_weights(), net1.get_weights()
    assert np.abs(w1 - w0).max() <= 1e-2 * np.abs(w0).max()
    with pytest.raises(hisq.HisqError):
        hisq.Net.trained(ctx, B[:0], X[:0])


def test_residual_loss_and_gradient_match_oracle(small):
    dims, ctx, fat, lng = small
    m = 0.1
    net = hisq.Net(ctx, loss=1, mass=m)
    chans = [1, 8, 8, 8, 1]
    w = rand_weights(chans, 9)
    net.set_weights(w)
    b = fields.gaussian_source(dims, 303)[0]
    x = fields.gaussian_source(dims, 304)[0]
    loss, g = net.loss_grad(b.cuda(), x.cuda())
    loss_o, g_o = oracle.net_loss_grad_residual(dims, fat, lng, chans, w, b.numpy(), x.numpy(), m)
    assert abs(loss - loss_o) <= TOL_FWD[1] * loss_o
    check_gradient(g, g_o, chans)


def test_residual_loss_training_lowers_fcg_iterations():
    # trained on the residual norm |A (K b - x)|^2 / |b|^2, the network takes flexible CG to
    # the FP64 residual 1e-10 in fewer iterations than flexible CG with K = identity (= CG)
    dims, m = (8, 8, 8, 8), 0.05
    fat, lng = fields.recipe_links(dims, 0.5, 77)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F64X, hisq.F32, hisq.F16))
    npairs = 64
    B = fields.gaussian_source(dims, 310, npairs).cuda()
    X = torch.zeros_like(B)
    for k in range(0, npairs, 16):
        rc, st = ctx.cg(m, B[k:k + 16].contiguous(), X[k:k + 16], tol=1e-8, prec_sloppy=hisq.F32,
                        prec_precise=hisq.F64)
        assert rc == hisq.OK
    net = hisq.Net(ctx, epochs=6, batch=8, lr=3e-3, loss=1, mass=m)
    losses = net.train(B, X, 6)
    assert np.all(np.isfinite(losses)) and losses[-1] < 0.5 * losses[0]
    its_net, its_id = [], []
    for i in range(3):
        b = fields.gaussian_source(dims, 900 + i)[0]
        x = torch.zeros_like(b).cuda()
        rc, st = hisq.fcg(ctx, m, b.cuda(), x, net=net, tol=1e-10, prec_precise=hisq.F64X)
        assert rc == hisq.OK and st.reliable_updates == 0  # the network was kept throughout
        r = b.numpy() - oracle.mdagm(dims, fat.numpy(), lng.numpy(), m, x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(b.numpy()) <= 1e-10
        its_net.append(st.iterations)
        rc0, st0 = hisq.fcg(ctx, m, b.cuda(), torch.zeros_like(b).cuda(), net=None, tol=1e-10, prec_precise=hisq.F64X)
        its_id.append(st0.iterations)
    print(f"residual-loss training: losses {losses}, FCG(net) {its_net}, FCG(identity) {its_id}")
    assert max(its_net) < 0.9 * min(its_id)


def test_network_may_outlive_its_context():
    dims = (6, 4, 4, 6)
    fat, lng = fields.recipe_links(dims, 0.5, 78)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F32))
    net = hisq.Net(ctx, link_prec=hisq.F32)
    ctx.close()
    net.close()
    torch.cuda.synchronize()
    assert float(torch.ones(4, device="cuda").sum()) == 4.0


def test_bounded_wait_error_reaches_the_host():
    # the tensor-core layer's barrier waits are bounded: with the self-test option every layer
    # launch first waits on a barrier that nothing completes; the wait runs out (about 1 ms),
    # the kernel raises the context's device error flag and skips its output, and the next
    # synchronising call returns HISQ_EDEVICE.  The context stays usable afterwards.
    dims = (6, 4, 4, 6)
    fat, lng = fields.recipe_links(dims, 0.5, 80)
    ctx = hisq.Context(dims, fat.cuda(), lng.cuda(), precs=(hisq.F64, hisq.F32, hisq.F16))
    net = hisq.Net(ctx, selftest_wait=1)
    b = fields.gaussian_source(dims, 340)[0].cuda()
    x = fields.gaussian_source(dims, 341)[0].cuda()
    with pytest.raises(hisq.HisqError) as err:
        net.loss_grad(b, x)
    assert err.value.code == hisq.EDEVICE
    net.close()
    # the same context still computes correct results
    out = torch.empty_like(b)
    ctx.dslash(0, b, out)
    want = oracle.dslash(dims, fat.numpy(), lng.numpy(), b.cpu().numpy(), 0)
    assert np.abs(out.cpu().numpy() - want).max() <= 1e-13 * np.abs(want).max()
    good = hisq.Net(ctx)
    good.loss_grad(b, x)
    good.close()
    ctx.close()


def test_tensor_core_network_full_size_vs_oracle():
    # The 32^3 x 8 workload of the learned preconditioner (16-bit links, eps 0.5): the two
    # 8 -> 8 layers have 2048 tiles of 128 sites and run on persistent CTAs, at most
    # (resident CTAs per SM) x 152 of them, so every CTA handles two or three tiles in turn,
    # carrying its mbarrier phases and reusing its TMEM accumulator from tile to tile.  The
    # whole output is compared with the oracle's FP64 network, norm-wise and per block of
    # 128 consecutive output sites (a tile computed with a stale phase or accumulator would
    # stand out in the blocks it reaches).
    dims = (32, 32, 32, 8)
    fat, lng = fields.recipe_links(dims, 0.5, 1003, device="cuda")
    ctx = hisq.Context(dims, fat, lng, precs=(hisq.F16,))
    fh, lh = fat.cpu().numpy(), lng.cpu().numpy()
    del fat, lng
    chans = [1, 8, 8, 8, 1]
    w = rand_weights(chans, 21)
    outs = {}
    b = fields.gaussian_source(dims, 350)[0]
    for tc in (1, 0):
        net = hisq.Net(ctx, link_prec=hisq.F16, tensor_cores=tc)
        net.set_weights(w)
        z = torch.full_like(b, float("nan")).cuda()
        net.apply(b.cuda(), z)
        outs[tc] = z.cpu().numpy()
        net.close()
    want = oracle.net_apply(dims, fh, lh, chans, w, b.numpy())
    for tc in (1, 0):
        got = outs[tc]
        assert np.isfinite(got).all()
        e = rel(got, want)
        assert e <= TOL_FWD[tc], (tc, e)
        blk = np.linalg.norm((got - want).reshape(-1, 128 * 3), axis=1) / np.linalg.norm(want.reshape(-1, 128 * 3),
                                                                                          axis=1)
        assert blk.max() <= 1.25 * TOL_FWD[tc], (tc, int(blk.argmax()), float(blk.max()))
        print(f"32^3x8 network, tensor cores {tc}: rel {e:.2e}, worst 128-site block {blk.max():.2e}")
    ctx.close()


def test_tensor_core_gradient_full_size_vs_oracle():
    # loss and weight gradient on the same 32^3 x 8 workload: the backward-data passes of the
    # 8 -> 8 layers run the persistent tensor-core kernel with conjugate re-indexed weights
    dims = (32, 32, 32, 8)
    fat, lng = fields.recipe_links(dims, 0.5, 1003, device="cuda")
    ctx = hisq.Context(dims, fat, lng, precs=(hisq.F16,))
    fh, lh = fat.cpu().numpy(), lng.cpu().numpy()
    del fat, lng
    chans = [1, 8, 8, 8, 1]
    w = rand_weights(chans, 22)
    net = hisq.Net(ctx, link_prec=hisq.F16, tensor_cores=1)
    net.set_weights(w)
    b = fields.gaussian_source(dims, 351)[0]
    x = fields.gaussian_source(dims, 352)[0]
    loss, g = net.loss_grad(b.cuda(), x.cuda())
    loss_o, g_o = oracle.net_loss_grad(dims, fh, lh, chans, w, b.numpy(), x.numpy())
    assert abs(loss - loss_o) <= TOL_FWD[1] * loss_o
    check_gradient(g, g_o, chans)
    net.close()
    ctx.close()
