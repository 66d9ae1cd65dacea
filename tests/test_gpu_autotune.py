"""Autotuner on the GPU: every candidate launch shape (pipelined or plain first
transform pass, RAHT tile 256..1024, transform and prelude grid sizes) gives byte-identical bitstreams and decoded
frames, the best setting is applied and cached, and a cache hit reapplies it."""
import numpy as np
import pytest

from paper_2606_05650_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05650_gb300 import gsnfs
    yield gsnfs
    for k in gsnfs.TUNABLES:
        gsnfs.tune_set(k, 0)


def test_every_launch_shape_gives_identical_outputs(G, tmp_path):
    from paper_2606_05650_gb300 import autotune
    frames = [syn.DynamicScene(40).frame(t, n=n) for t, n in enumerate([150_000, 60_000])]
    P = [torch.from_numpy(p).cuda() for p, _ in frames]
    A = [torch.from_numpy(a).cuda() for _, a in frames]
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    cache = str(tmp_path / "tune.json")
    e = autotune.tune_round_trip(P, A, [16, 17], qp, reps=1, cache=cache)
    ran = [t for t in e["trials"] if t[1] is not None]
    assert len(ran) == len(e["trials"]) >= 11
    assert all(ok for _, _, ok in ran), e["trials"]
    assert {k: G.tune_get(k) for k in G.TUNABLES} == e["params"]
    for k in G.TUNABLES:
        G.tune_set(k, 0)
    hit = autotune.tune_round_trip(P, A, [16, 17], qp, cache=cache)
    assert hit["cached"] and {k: G.tune_get(k) for k in G.TUNABLES} == e["params"]


def test_tunable_validation(G):
    with pytest.raises(G.GsnfsError):
        G.tune_set("raht_tile", 300)
    with pytest.raises(G.GsnfsError):
        G.tune_set("raht_grid", 33)
    with pytest.raises(G.GsnfsError):
        G.tune_set("raht_pipe", 3)
    G.tune_set("raht_tile", 4096)
    assert G.tune_get("raht_tile") == 4096
    G.tune_set("raht_tile", 0)


def test_extreme_tiles_give_identical_streams(G):
    p, a = syn.DynamicScene(41).frame(0, n=50_000)
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    pd, ad = torch.from_numpy(p).cuda(), torch.from_numpy(a).cuda()
    ref, nv, rp, ra = G.encode_frame(pd, ad, 16, qp, recon=True)
    ref = ref.cpu().numpy()
    ra = ra.cpu().numpy()
    for tile, grid, pgrid, plain in ((4096, 1, 1, 0), (256, 32, 32, 1), (2048, 0, 2, 0), (0, 0, 0, 1), (0, 0, 0, 2)):
        G.tune_set("raht_tile", tile)
        G.tune_set("raht_grid", grid)
        G.tune_set("prelude_grid", pgrid)
        G.tune_set("raht_pipe", plain)
        got, _, _, ga = G.encode_frame(pd, ad, 16, qp, recon=True)
        assert np.array_equal(got.cpu().numpy(), ref), tile
        assert np.array_equal(ga.cpu().numpy(), ra), tile
        dp, da = G.decode_frame(got)
        assert np.array_equal(da.cpu().numpy(), ra), tile
    for k in G.TUNABLES:
        G.tune_set(k, 0)
