"""The persistent tile-queue inverse (variant 5, n = 256, xi output): the same bits as the fused register
tile (variant 3, which the oracle pins) at the benchmark's full size and over repeated calls and graph
replays (its queue counters reset themselves), for several counts of source parameters (the split of the
dependency into two halves of q) and with per-band alpha; and its bounded waits: with the column tiles'
releases withheld, the row tiles' waits run out, the call returns with FR3D_INFO_TIMEOUT, and the next
call is exact again."""

import time

import pytest

from paper_1703_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    from paper_1703_01216_gb300 import build, fr3d
    assert torch.cuda.is_available()
    build.build()
    fr3d.load()
    prev = fr3d.autotune_mode()
    yield fr3d
    fr3d.autotune_mode(prev)
    fr3d.test_withhold_queue_counts(False)


def _data(F, w):
    H = F.kernel_transform(w.n, w.x0, w.h, w.zr, w.zy, w.nu)
    zeta = torch.empty((w.Q, w.Mp, w.n, w.n), device="cuda")
    F.zeta_from_xi(H, torch.as_tensor(w.xi_true, dtype=torch.float32, device="cuda"), w.sources, zeta)
    U = torch.empty((w.Q, 1, w.n, w.n), device="cuda")
    F.fwd_apply(H, zeta, w.Q, U)
    nz = torch.as_tensor(w.noise, dtype=torch.float32, device="cuda")
    nz *= w.noise_level * U.norm() / nz.norm()
    return H, U + nz, float(nz.norm())


def _run(F, H, U, q, w, delta, variant, n_bands=1, info=None):
    F.autotune_mode(2 + variant)
    out = torch.full((w.Mp, w.n, w.n), float("nan"), device="cuda")
    idx = torch.zeros(max(1, n_bands), dtype=torch.int32, device="cuda")
    F.invert(H, U, q, out, F.Opts(alphas=w.alphas, delta=delta, tau=1.1, points=w.sources, alpha_idx=idx,
                                  n_bands=n_bands, info=info))
    assert F.autotune_query(H)[0] == variant
    return out, idx


def test_full_size_matches_the_register_tile_over_repeated_calls(F):
    w = I.config_workload(3)
    H, U, delta = _data(F, w)
    ref, ridx = _run(F, H, U, w.Q, w, delta, 3)
    for _ in range(3):
        got, gidx = _run(F, H, U, w.Q, w, delta, 5)
        assert torch.equal(gidx, ridx)
        assert torch.equal(got, ref)


@pytest.mark.parametrize("q", [1, 2, 3, 5])
@pytest.mark.parametrize("n_bands", [1, 4])
def test_source_counts_and_bands_match_the_register_tile(F, q, n_bands):
    w = I.make_workload(256, 5, q=q, n_incl=3, noise_level=0.02, n_alpha=12, seed=900 + q)
    H, U, delta = _data(F, w)
    ref, ridx = _run(F, H, U, q, w, delta, 3, n_bands=n_bands)
    got, gidx = _run(F, H, U, q, w, delta, 5, n_bands=n_bands)
    assert torch.equal(gidx, ridx)
    assert torch.equal(got, ref)


def test_graph_replays_are_exact(F):
    w = I.make_workload(256, 40, q=4, n_incl=3, noise_level=0.02, n_alpha=12, seed=950)
    H, U, delta = _data(F, w)
    ref, _ = _run(F, H, U, 4, w, delta, 3)
    F.autotune_mode(2 + 5)
    out = torch.full_like(ref, float("nan"))
    opts = F.Opts(alphas=w.alphas, delta=delta, tau=1.1, points=w.sources)
    F.invert(H, U, 4, out, opts)            # allocates the queue's buffers outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            F.invert(H, U, 4, out, opts)
    torch.cuda.current_stream().wait_stream(st)
    for _ in range(3):
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_withheld_releases_end_in_a_timeout_report_and_the_next_call_is_exact(F):
    w = I.make_workload(256, 6, q=2, n_incl=2, noise_level=0.02, n_alpha=12, seed=970)
    H, U, delta = _data(F, w)
    ref, _ = _run(F, H, U, 2, w, delta, 3)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    F.test_withhold_queue_counts(True)
    try:
        t0 = time.perf_counter()
        _run(F, H, U, 2, w, delta, 5, info=info)
        torch.cuda.synchronize()
        assert time.perf_counter() - t0 < 30.0
    finally:
        F.test_withhold_queue_counts(False)
    assert int(info.item()) & F.INFO_TIMEOUT
    info.zero_()
    got, _ = _run(F, H, U, 2, w, delta, 5, info=info)
    torch.cuda.synchronize()
    assert not int(info.item()) & F.INFO_TIMEOUT
    assert torch.equal(got, ref)


def test_many_repeats_and_random_counts_match_the_register_tile(F):
    """The queue's ordering is timing-dependent (tickets, per-depth counters, bulk copies): repeat the
    full-size call, directly and as graph replays, and draw source, depth and band counts at random."""
    import random
    w = I.config_workload(3)
    H, U, delta = _data(F, w)
    ref, _ = _run(F, H, U, w.Q, w, delta, 3)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    F.autotune_mode(2 + 5)
    out = torch.empty_like(ref)
    opts = F.Opts(alphas=w.alphas, delta=delta, tau=1.1, points=w.sources, info=info)
    for _ in range(40):
        out.fill_(float("nan"))
        F.invert(H, U, w.Q, out, opts)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        assert not int(info.item()) & F.INFO_TIMEOUT
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            F.invert(H, U, w.Q, out, opts)
    torch.cuda.current_stream().wait_stream(st)
    for _ in range(40):
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    rnd = random.Random(11)
    for case in range(8):
        q, mp, nb = rnd.randint(1, 8), rnd.choice([1, 3, 7, 16, 33, 64]), rnd.choice([1, 4])
        w2 = I.make_workload(256, mp, q=q, n_incl=2, noise_level=0.02, n_alpha=12, seed=3100 + case)
        H2, U2, d2 = _data(F, w2)
        r, ri = _run(F, H2, U2, q, w2, d2, 3, n_bands=nb)
        for _ in range(3):
            got, gi = _run(F, H2, U2, q, w2, d2, 5, n_bands=nb)
            assert torch.equal(gi, ri), (q, mp, nb)
            assert torch.equal(got, r), (q, mp, nb)
        H2.close()
