"""Solvers on a non-blocking stream (a torch side stream) compute exactly what they compute
on the legacy default stream, also when their device memory is recycled from a solver that
was just destroyed (the buffers are zeroed on the solver's own stream, so no zeroing can land
after the solver's first kernels)."""
import numpy as np
import pytest
import torch

from paper_2003_08746_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jz():
    from paper_2003_08746_gb300 import build, jz as J
    build.build()
    J.load()
    assert torch.cuda.is_available()
    return J


@pytest.mark.parametrize("prec_name", ["JZ_PREC_FP64", "JZ_PREC_FP32FLUX"])
def test_side_stream_after_destroy_matches_default_stream(jz, prec_name):
    prec = getattr(jz, prec_name)
    g = W.jet_grid(256, 256, 128)
    q = torch.from_numpy(W.jet_state(g)).cuda()
    prm = W.jet_params(seed=2)
    grid = jz.Grid.from_workload(g)
    ref = jz.Solver(grid, prm, prec)
    ref.set_state(q, 0.0)
    st_ref = ref.step(2)
    q_ref = torch.empty_like(q)
    ref.get_state(q_ref)
    torch.cuda.synchronize()
    for trial in range(2):
        first = jz.Solver(grid, prm, jz.JZ_PREC_FP64 if trial == 0 else jz.JZ_PREC_FP32FLUX,
                          stream=torch.cuda.Stream().cuda_stream)
        first.set_state(q, 0.0)
        first.step(1, stats=False)
        first.close()                           # its memory goes back to the driver
        side = torch.cuda.Stream()
        s = jz.Solver(grid, prm, prec, stream=side.cuda_stream)
        s.set_state(q, 0.0)
        st = s.step(2)
        out = torch.empty_like(q)
        s.get_state(out)
        side.synchronize()
        assert st.t == st_ref.t and st.min_p == st_ref.min_p
        assert torch.equal(out, q_ref), f"trial {trial}: max diff {(out - q_ref).abs().max().item()}"
        s.close()


def test_adjoint_on_side_stream(jz):
    g = W.jet_grid(32, 24, 16)
    prm = W.jet_params(seed=4)
    q = W.jet_state(g)
    grid = jz.Grid.from_workload(g)
    A = np.asarray(prm.forcing_amp)
    a = jz.Solver(grid, prm)
    a.set_state(q, 0.0)
    Ja, ga = jz.jz_adjoint_step(a.h, A, 6, 3, 0.75)
    side = torch.cuda.Stream()
    b = jz.Solver(grid, prm, stream=side.cuda_stream)
    b.set_state(q, 0.0)
    Jb, gb = jz.jz_adjoint_step(b.h, A, 6, 3, 0.75)
    # J and dJ/dA are sums with atomic additions: equal up to the order of those sums
    assert abs(Ja - Jb) <= 1e-12 * abs(Ja)
    assert np.abs(ga - gb).max() <= 1e-12 * np.abs(ga).max()


def test_state_transfer_paths_agree(jz):
    """jz_set_state / jz_get_state from and to device memory, page-locked host memory (read
    and written by the packing kernels over the host link) and pageable host memory (staging
    copy) move the same bytes."""
    g = W.jet_grid(70, 34, 16)
    q = W.jet_state(g) + 1e-3 * np.random.default_rng(3).standard_normal((5, g.nk, g.nj, g.ni))
    prm = W.jet_params(seed=2)
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP64, stream=torch.cuda.Stream().cuda_stream)
    sources = {"pageable": q, "pinned": torch.from_numpy(q).pin_memory(), "device": torch.from_numpy(q).cuda()}
    outs = {}
    for name, src in sources.items():
        s.set_state(src, 0.0)
        s.step(1, stats=False)
        for oname, dst in (("pageable", np.empty_like(q)), ("pinned", torch.empty(q.shape, dtype=torch.float64).pin_memory()),
                           ("device", torch.empty(q.shape, dtype=torch.float64, device="cuda"))):
            s.get_state(dst)
            torch.cuda.synchronize()
            outs[(name, oname)] = dst.cpu().numpy() if isinstance(dst, torch.Tensor) else dst
    ref = outs[("pageable", "pageable")]
    for key, val in outs.items():
        assert np.array_equal(val, ref), key


@pytest.mark.parametrize("prec_name", ["JZ_PREC_FP64", "JZ_PREC_FP32FLUX"])
def test_step_graphs_match_plain_launches(jz, prec_name):
    """jz_rk_step replays pairs of steps as a CUDA graph; with profiling on it launches every
    kernel itself.  Both give the same bits, for even and odd step counts, across calls and
    after jz_set_state."""
    prec = getattr(jz, prec_name)
    g, q, prm = W.make_workload("box32x24x16")
    grid = jz.Grid.from_workload(g)
    plain = jz.Solver(grid, prm, prec)
    plain.profile(True)                          # events between kernels: no graphs
    graph = jz.Solver(grid, prm, prec, stream=torch.cuda.Stream().cuda_stream)
    for s in (plain, graph):
        s.set_state(q, 0.0)
    for n in (1, 4, 7, 2):
        a, b = plain.step(n), graph.step(n)
        assert a.t == b.t and a.steps == b.steps
        assert np.array_equal(plain.get_state(), graph.get_state()), n
    for s in (plain, graph):
        s.set_state(q, 0.0)
    a, b = plain.step(6), graph.step(6)
    assert np.array_equal(plain.get_state(), graph.get_state()) and a.t == b.t
