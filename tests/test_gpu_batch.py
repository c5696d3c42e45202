"""Batches of independent precision-form matrices of uneven size (h2_batch_*),
through the C ABI.

Each member's result is checked against the quantized oracle (O-tree on the
member's dequantized blocks, FP64): only the FP32 accumulation differs, so the
relative l2 error stays within 2 u sqrt(N), N the member's longest FP32
accumulation (fp32_tol.py). The batch runs the same kernels as a single handle
over concatenated tables, so a member's result also agrees with that member's
own h2_matvec within twice that margin.
"""
import numpy as np
import pytest

import h2gen
import oracle
from oracle import quant
from fp32_tol import acc_tol, check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def h2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1902_01829_gb300 as mod

    return mod


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda().t()


def nan_like(n, nv):
    return torch.full((nv, n), float("nan"), dtype=torch.float64, device="cuda").t()


# uneven members: log-uniform sizes plus the edge cases (one leaf, two leaves,
# a member skipped with nv = 0, a member with two passes of 16 vectors)
@pytest.fixture(scope="module")
def members():
    spec = h2gen.batch_workload(count=6, lo=9.5, hi=13.0, seed=41)
    spec += [(dict(dim=2, n=20, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=4101), 2),
             (dict(dim=2, n=61, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=4102), 1),
             (dict(dim=2, n=3001, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=4103), 0),
             (dict(dim=2, n=2500, m=32, p=4, eta=0.9, kernel="exp", ell=0.1, seed=4104), 20)]
    return [(h2gen.generate(**kw), nv) for kw, nv in spec]


def _check_members(mats, xs, ys, form, bases_fp32):
    for (A, nv), x, y in zip(mats, xs, ys):
        if nv == 0:
            assert torch.isnan(y).all()  # untouched
            continue
        got = y.cpu().numpy()
        ref = oracle.matvec(A, x, **quant.dequantized_arrays(A, form, bases_fp32))
        check(oracle.rel_l2(got, ref), acc_tol(A), ("member", A.n, nv, form, bases_fp32))


@pytest.mark.parametrize("form,bases_fp32", [("fp16", False), ("int16", True), ("bf16", False), ("fp16", True)])
def test_batch_matches_quantized_oracle(h2, members, form, bases_fp32):
    Ms = [h2.H2Matrix.from_generator(A, storage=form, bases_fp32=bases_fp32) for A, _ in members]
    B = h2.H2Batch(Ms)
    info = B.info()
    assert info["members"] == len(members)
    assert info["coupling_rows"] == sum(A.n_nodes for A, _ in members)
    xs_np = [h2gen.vectors(700 + i, A.n, max(nv, 1)) for i, (A, nv) in enumerate(members)]
    xs = [to_dev(x) if nv else None for x, (_, nv) in zip(xs_np, members)]
    ys = [nan_like(A.n, max(nv, 1)) for A, nv in members]
    B.matvec(xs, ys)
    B.check()
    _check_members(members, [x[:, :max(nv, 1)] for x, (_, nv) in zip(xs_np, members)], ys, form, bases_fp32)
    # each member alone (h2_matvec) agrees with its batched result
    for (A, nv), M, x, y in zip(members, Ms, xs, ys):
        if nv:
            alone = M.matvec(x).cpu().numpy()
            check(oracle.rel_l2(y.cpu().numpy(), alone), 2 * acc_tol(A), ("batched vs alone", A.n, nv))
    B.close()
    for M in Ms:
        M.close()


@pytest.mark.parametrize("form", ["fp16", "bf16"])
def test_batch_of_k64_members_with_panel_coupling(h2, form):
    """k = 64 members keep their coupling codes in the panel layout (the tensor-core operand layout);
    the batch reads them on the CUDA cores, for every member's vector count."""
    mats = [(h2gen.generate(dim=3, n=4096, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=4201), 16),
            (h2gen.generate(dim=3, n=2500, m=64, p=4, eta=0.8, kernel="matern32", ell=0.2, seed=4202), 3)]
    Ms = [h2.H2Matrix.from_generator(A, storage=form) for A, _ in mats]
    B = h2.H2Batch(Ms)
    xs_np = [h2gen.vectors(720 + i, A.n, nv) for i, (A, nv) in enumerate(mats)]
    xs = [to_dev(x) for x in xs_np]
    ys = [nan_like(A.n, nv) for A, nv in mats]
    B.matvec(xs, ys)
    B.check()
    _check_members(mats, xs_np, ys, form, False)
    B.close()
    for M in Ms:
        M.close()


def test_batch_repeated_calls_and_new_buffers(h2, members):
    Ms = [h2.H2Matrix.from_generator(A, storage="fp16") for A, _ in members]
    B = h2.H2Batch(Ms)
    for rep in range(3):  # new vectors in new buffers each time: the pointer table is rewritten per call
        nvs = [(nv + rep) % 5 for _, nv in members]
        xs_np = [h2gen.vectors(800 + 10 * rep + i, A.n, max(nv, 1)) for i, ((A, _), nv) in enumerate(zip(members, nvs))]
        xs = [to_dev(x) if nv else None for x, nv in zip(xs_np, nvs)]
        ys = [nan_like(A.n, max(nv, 1)) for (A, _), nv in zip(members, nvs)]
        B.matvec(xs, ys)
        B.check()
        _check_members([(A, nv) for (A, _), nv in zip(members, nvs)], xs_np, ys, "fp16", False)
    B.close()


def test_batch_of_one_equals_handle(h2, members):
    A, _ = members[0]
    M = h2.H2Matrix.from_generator(A, storage="int16", bases_fp32=True)
    B = h2.H2Batch([M])
    x = to_dev(h2gen.vectors(901, A.n, 3))
    y = nan_like(A.n, 3)
    B.matvec([x], [y])
    B.check()
    check(oracle.rel_l2(y.cpu().numpy(), M.matvec(x).cpu().numpy()), 2 * acc_tol(A), "batch of one vs handle")
    B.close()
    M.close()


def test_batch_graph_capture_replays_with_new_inputs(h2, members):
    Ms = [h2.H2Matrix.from_generator(A, storage="fp16") for A, _ in members]
    B = h2.H2Batch(Ms)
    nvs = [max(nv, 1) for _, nv in members]
    xs = [torch.zeros((nv, A.n), dtype=torch.float64, device="cuda").t() for (A, _), nv in zip(members, nvs)]
    ys = [torch.zeros_like(x) for x in xs]
    args = B.prepare(xs, ys)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        B.matvec_prepared(args, s)  # first product before capture (kernel attributes are set once)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        B.matvec_prepared(args, s)
    for rep in range(2):
        xs_np = [h2gen.vectors(950 + 10 * rep + i, A.n, nv) for i, ((A, _), nv) in enumerate(zip(members, nvs))]
        for x, xn in zip(xs, xs_np):
            x.copy_(to_dev(xn))
        for y in ys:
            y.fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        B.check()
        _check_members([(A, nv) for (A, _), nv in zip(members, nvs)], xs_np, ys, "fp16", False)
    del g
    B.close()


def test_batch_rejects_bad_members_and_arguments(h2, members):
    A0, A1 = members[0][0], members[1][0]
    f16 = h2.H2Matrix.from_generator(A0, storage="fp16")
    i16 = h2.H2Matrix.from_generator(A1, storage="int16")
    f64 = h2.H2Matrix.from_generator(A1, storage="fp64")
    f16b = h2.H2Matrix.from_generator(A1, storage="fp16", bases_fp32=True)
    for mats, status in (([f64], h2.H2_ERR_UNSUPPORTED), ([f16, i16], h2.H2_ERR_INVALID),
                         ([f16, f16], h2.H2_ERR_INVALID), ([f16, f16b], h2.H2_ERR_INVALID)):
        with pytest.raises(h2.H2Error) as ei:
            h2.H2Batch(mats)
        assert ei.value.status == status, str(ei.value)
    B = h2.H2Batch([f16])
    x = to_dev(h2gen.vectors(990, A0.n, 2))
    y = torch.zeros_like(x)
    nv, xp, ldx, yp, ldy = B.prepare([x], [y])
    ldx[0] = A0.n - 1
    with pytest.raises(h2.H2Error) as ei:
        B.matvec_prepared((nv, xp, ldx, yp, ldy))
    assert ei.value.status == h2.H2_ERR_INVALID
    nv[0] = -1
    with pytest.raises(h2.H2Error) as ei:
        B.matvec_prepared((nv, xp, ldx, yp, ldy))
    assert ei.value.status == h2.H2_ERR_INVALID
    B.close()
    for M in (f16, i16, f64, f16b):
        M.close()


@pytest.mark.slow
def test_full_batch_sampled_members(h2):
    """The full batched workload (256 members, n log-uniform in [2^12, 2^17], nv in {1, 4, 16}) in
    the launch configuration the benchmark times; the smallest, the largest and two other members
    are compared with the quantized oracle, and every member's result is finite."""
    spec = h2gen.batch_workload()
    Ms, nvs, xs, ys, keep = [], [], [], [], {}
    ns = [kw["n"] for kw, _ in spec]
    sample = {int(np.argmin(ns)), int(np.argmax(ns)), 17, 201}
    for i, (kw, nv) in enumerate(spec):
        A = h2gen.generate(**kw)
        Ms.append(h2.H2Matrix.from_generator(A, storage="fp16"))
        x = h2gen.vectors(5000 + i, A.n, nv)
        xs.append(to_dev(x))
        ys.append(nan_like(A.n, nv))
        nvs.append(nv)
        if i in sample:
            keep[i] = (A, x)
        else:
            A.free()
    B = h2.H2Batch(Ms)
    B.matvec(xs, ys)
    B.check()
    for y in ys:
        assert torch.isfinite(y).all()
    for i, (A, x) in keep.items():
        ref = oracle.matvec(A, x, **quant.dequantized_arrays(A, "fp16"))
        check(oracle.rel_l2(ys[i].cpu().numpy(), ref), acc_tol(A), ("sampled member", i, A.n, nvs[i]))
    B.close()
    for M in Ms:
        M.close()


def test_batch_tune_chooses_a_candidate_and_keeps_the_products(h2, members):
    Ms = [h2.H2Matrix.from_generator(A, storage="fp16") for A, _ in members]
    B = h2.H2Batch(Ms)
    xs_np = [h2gen.vectors(990 + i, A.n, max(nv, 1)) for i, (A, nv) in enumerate(members)]
    xs = [to_dev(x) if nv else None for x, (_, nv) in zip(xs_np, members)]
    ys = [nan_like(A.n, max(nv, 1)) for A, nv in members]
    chosen = B.tune(xs, ys)
    assert chosen["consumer_warps"] in (8, 16) and chosen["chunk_blocks"] in (64, 128, 256)
    assert chosen["tree_leaves"] in (16, 32, 64)
    ys = [nan_like(A.n, max(nv, 1)) for A, nv in members]
    B.matvec(xs, ys)
    B.check()
    _check_members(members, xs_np, ys, "fp16", False)
    B.close()
