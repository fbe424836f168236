"""Batched transforms of fields with uneven sizes (one ABCD per field): the
persistent per-pass launches and their captured CUDA graph against per-field
launches and against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import nslct_oracle as O
from paper_1707_03688_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SIZES = [64, 96, 128, 192, 256, 384, 512, 768, 1024]


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_03688_gb300 import build as B
    B.build()
    from paper_1707_03688_gb300 import nslct
    nslct.load()
    return nslct


@pytest.fixture(scope="module")
def batch_case(N):
    rng = np.random.default_rng(3)
    shapes = [(int(rng.choice(SIZES)), int(rng.choice(SIZES))) for _ in range(24)]
    shapes[0] = (64, 1024)   # extremes included
    shapes[1] = (1024, 64)
    abcds = [I.random_symplectic_abcd(3000 + k) for k in range(len(shapes))]
    fields = [I.blob_field(nx, ny, seed=3100 + k, width_range=(2.0, max(3.0, min(nx, ny) / 8)))
              for k, (nx, ny) in enumerate(shapes)]
    b = N.Batch(abcds, shapes)
    ins = [torch.from_numpy(f).to(torch.complex64).cuda() for f in fields]
    outs = [torch.empty_like(x) for x in ins]
    b.bind(ins, outs)
    return b, shapes, abcds, fields, ins, outs


def test_batch_matches_single_plans_and_oracle(N, batch_case):
    b, shapes, abcds, fields, ins, outs = batch_case
    b.forward()
    torch.cuda.synchronize()
    for k, (nx, ny) in enumerate(shapes):
        plan = N.Plan(abcds[k], nx, ny)
        ref = plan.forward(ins[k])
        torch.cuda.synchronize()
        got = outs[k].cpu().numpy().astype(np.complex128)
        single = ref.cpu().numpy().astype(np.complex128)
        assert O.rel_l2(got, single) < 2e-6, (k, nx, ny)
        # the batch's own plan for this field equals a standalone plan
        np.testing.assert_allclose(b.params(k)["H"], plan.params()["H"], atol=0)
        params = O.decompose(b.info(k)["abcd"], b.params(k)["H"])
        ref_o = O.forward(fields[k], params, b.dx[k], b.dy[k])
        assert O.rel_l2(got, ref_o) < 2e-5, (k, nx, ny)
        plan.close()


def test_batch_graph_and_each_agree(N, batch_case):
    b, shapes, abcds, fields, ins, outs = batch_case
    b.forward()
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    # run again: counters are reset every run
    b.forward()
    torch.cuda.synchronize()
    for a, o in zip(first, outs):
        assert torch.equal(a, o)
    # graph capture replays the same launches
    s = torch.cuda.Stream()
    b.capture(s)
    for o in outs:
        o.zero_()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        b.forward(stream=s)
    s.synchronize()
    for a, o in zip(first, outs):
        assert torch.equal(a, o)
    # per-field launches through the single-field kernels
    b.forward_each()
    torch.cuda.synchronize()
    for a, o in zip(first, outs):
        assert O.rel_l2(o.cpu().numpy().astype(np.complex128), a.cpu().numpy().astype(np.complex128)) < 2e-6


def test_batch_pass_sequence_equals_forward(N, batch_case):
    """Passes 0..4 enqueued one by one give nslct_batch_forward's outputs
    exactly, with every field batched and with the large ones run alone."""
    b, shapes, abcds, fields, ins, outs = batch_case
    for split in (1 << 30, 512):
        b.set_split(split)
        b.forward()
        torch.cuda.synchronize()
        ref = [o.clone() for o in outs]
        for o in outs:
            o.zero_()
        for k in range(5):
            b.forward_pass(k)
        torch.cuda.synchronize()
        for k, (a, o) in enumerate(zip(ref, outs)):
            assert torch.equal(a, o), (split, k)
    with pytest.raises(N.NslctError) as exc:
        b.forward_pass(5)
    assert exc.value.code == N.NSLCT_E_ARG


def test_batch_cta_sizes_agree(N, batch_case):
    """Every batched CTA size, the packed 128-thread one included, gives the
    single-plan results; graph capture after pinning the size replays them."""
    b, shapes, abcds, fields, ins, outs = batch_case
    b.set_split(1 << 30)
    refs = []
    for k, (nx, ny) in enumerate(shapes):
        plan = N.Plan(abcds[k], nx, ny)
        refs.append(plan.forward(ins[k]).cpu().numpy().astype(np.complex128))
        plan.close()
    for th in (128, 256, 512):
        b.set_threads(th)
        assert b.threads == th
        for o in outs:
            o.zero_()
        b.forward()
        torch.cuda.synchronize()
        for k, (a, o) in enumerate(zip(refs, outs)):
            assert O.rel_l2(o.cpu().numpy().astype(np.complex128), a) < 2e-6, (th, k, shapes[k])
    b.set_threads(128)
    b.forward()
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    s = torch.cuda.Stream()
    b.capture(s)
    for o in outs:
        o.zero_()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        b.forward(stream=s)
    s.synchronize()
    for a, o in zip(first, outs):
        assert torch.equal(a, o)
    with pytest.raises(N.NslctError) as exc:
        b.set_threads(64)
    assert exc.value.code == N.NSLCT_E_ARG


LARGE_SHAPES = [(2048, 2048), (1536, 2048), (2048, 1536), (2048, 128), (128, 2048), (1536, 1536),
                (1536, 192), (768, 2048), (256, 384), (128, 128)]


@pytest.fixture(scope="module")
def large_case(N):
    """Fields with the 1536- and 2048-point lines of the 256-field workload,
    square and not, with their FP64 oracle outputs (computed once)."""
    abcds = [I.random_symplectic_abcd(3300 + k) for k in range(len(LARGE_SHAPES))]
    fields = [I.blob_field(nx, ny, seed=3400 + k, width_range=(2.0, max(3.0, min(nx, ny) / 8)))
              for k, (nx, ny) in enumerate(LARGE_SHAPES)]
    b = N.Batch(abcds, LARGE_SHAPES)
    ins = [torch.from_numpy(f).to(torch.complex64).cuda() for f in fields]
    outs = [torch.empty_like(x) for x in ins]
    b.bind(ins, outs)
    refs = []
    for k in range(len(LARGE_SHAPES)):
        params = O.decompose(b.info(k)["abcd"], b.params(k)["H"])
        refs.append(O.forward(fields[k], params, b.dx[k], b.dy[k]))
    yield b, refs, outs
    b.close()


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_batch_large_lines_match_oracle(N, large_case, threads):
    """Every field batched (no per-field passes), at each batched CTA size:
    each output against the oracle directly, 1536/2048-point lines included."""
    b, refs, outs = large_case
    b.set_split(1 << 30)
    b.set_threads(threads)
    for o in outs:
        o.zero_()
    b.forward()
    torch.cuda.synchronize()
    for k, (nx, ny) in enumerate(LARGE_SHAPES):
        err = O.rel_l2(outs[k].cpu().numpy().astype(np.complex128), refs[k])
        assert err < 2e-5, (threads, k, nx, ny, err)


def test_batch_rejects_unsupported_sizes(N):
    with pytest.raises(N.NslctError) as exc:
        N.Batch([I.random_symplectic_abcd(1)], [(48, 64)])
    assert exc.value.code == N.NSLCT_E_SIZE


def test_batch_split_and_tune(N, batch_case):
    """Fields at or above the split run through their own fused passes; the
    results agree with the all-batched run whatever the split, in direct
    launches and in a captured graph, and the tuner picks one of the sizes."""
    b, shapes, abcds, fields, ins, outs = batch_case
    b.set_split(1 << 30)
    b.forward()
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]

    def close_to_ref():
        for k, (a, o) in enumerate(zip(ref, outs)):
            assert O.rel_l2(o.cpu().numpy().astype(np.complex128), a.cpu().numpy().astype(np.complex128)) < 2e-6, k

    for split in (512, 96, 1):
        b.set_split(split)
        assert b.split == split
        for o in outs:
            o.zero_()
        b.forward()
        torch.cuda.synchronize()
        close_to_ref()
    s = torch.cuda.Stream()
    b.set_split(384)
    b.capture(s)
    for o in outs:
        o.zero_()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        b.forward(stream=s)
    s.synchronize()
    close_to_ref()
    chosen, ms = b.tune(iters=2)
    sizes = {min(nx, ny) for nx, ny in shapes} | {1 << 30}
    assert chosen in sizes and b.split == chosen and ms > 0 and b.threads in (128, 256, 512)
    for o in outs:
        o.zero_()
    b.forward()
    torch.cuda.synchronize()
    close_to_ref()
    b.set_split(1 << 30)


def test_batch_tune_rejects_in_place(N):
    shapes = [(64, 64), (128, 64)]
    b = N.Batch([I.random_symplectic_abcd(5 + k) for k in range(2)], shapes)
    xs = [torch.zeros(nx, ny, dtype=torch.complex64, device="cuda") for nx, ny in shapes]
    b.bind(xs, xs)
    with pytest.raises(N.NslctError) as exc:
        b.tune()
    assert exc.value.code == N.NSLCT_E_ARG
    b.close()
