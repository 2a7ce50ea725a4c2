"""Device memory of a hierarchy comes from the caller's allocator (GPU
required).  The binding passes PyTorch's caching allocator by default, so
every buffer a handle holds shows in torch.cuda.memory_allocated() and goes
back to torch when the handle is freed; results do not depend on where the
memory came from; an allocator that fails makes setup return an error with
every buffer it had handed out given back."""
import ctypes
import gc

import numpy as np
import pytest

import q1elasticity as q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

amg = pytest.importorskip("paper_2202_09056_gb300")

from parity_util import dev_args  # noqa: E402


def _allocated():
    """Bytes allocated through torch's caching allocator, after collecting
    garbage: tensors of an earlier test that a reference cycle (a caught
    exception's traceback) keeps alive would otherwise be freed in the middle
    of a measurement."""
    gc.collect()
    torch.cuda.synchronize()
    return torch.cuda.memory_allocated()


def test_hierarchy_lives_in_torch_memory_and_goes_back():
    p = q.make_problem((14, 12, 13), traction=(0, 0, -1), inclusion_frac=0.2)
    args = dev_args(p, torch)
    f = torch.from_numpy(p.f).cuda()
    base = _allocated()
    G = amg.AMG(*args, coarse_enough=300)          # default: torch's caching allocator
    held = _allocated() - base
    st = G.stats()
    assert st["bytes_total"] >= st["bytes_matrices"] > 0
    # torch rounds each block up to 512 bytes
    assert st["bytes_total"] <= held <= 1.05 * st["bytes_total"] + (1 << 20), (held, st)
    u, it, res, s = G.solve(f)
    after_solve = _allocated() - base
    assert after_solve == held + (u.numel() * 8 + 511) // 512 * 512  # the solve allocates only u
    # the same hierarchy on the library's own allocations gives the same bits
    G2 = amg.AMG(*args, coarse_enough=300, allocator=None)
    assert _allocated() - base == after_solve
    u2, it2, res2, s2 = G2.solve(f)
    assert (it, res, s) == (it2, res2, s2) and torch.equal(u, u2)
    del u, u2
    G.close()
    G2.close()
    assert _allocated() == base


def test_batch_lives_in_torch_memory():
    mats, Bs, F = [], [], []
    for shape in ((6, 5, 7), (8, 8, 8)):
        p = q.make_problem(shape, body=(0, 0, -1))
        rp, cl, val, B = dev_args(p, torch)
        mats.append((rp, cl, val))
        Bs.append(B)
        F.append(torch.from_numpy(np.atleast_2d(p.f).copy()).cuda())
    base = _allocated()
    bat = amg.AMGBatch(mats, Bs, [1, 1], coarse_enough=100)
    assert _allocated() - base >= bat.info()["bytes_total"] > 0
    U, its, res, st = bat.solve(F)
    assert st == amg.AMG_OK
    del U
    bat.close()
    assert _allocated() == base


class _Failing:
    """An allocator on torch's memory that returns NULL from its k-th call on."""

    def __init__(self, k):
        self.k, self.calls, self.live = k, 0, {}
        self.struct = amg.Allocator(amg._ALLOC_FN(self._alloc), amg._FREE_FN(self._free), None)

    def _alloc(self, ctx, n, stream):
        self.calls += 1
        if self.calls >= self.k:
            return None
        ptr = int(torch.cuda.caching_allocator_alloc(int(n), stream=int(stream or 0)))
        self.live[ptr] = n
        return ptr

    def _free(self, ctx, ptr, n, stream):
        assert self.live.pop(int(ptr)) == n
        torch.cuda.caching_allocator_delete(int(ptr))


@pytest.mark.parametrize("k", [1, 5, 40])
def test_failing_allocator_is_an_error_and_leaks_nothing(k):
    p = q.make_problem((9, 8, 10), traction=(0, 0, -1), inclusion_frac=0.2)
    args = dev_args(p, torch)
    base = _allocated()
    fa = _Failing(k)
    with pytest.raises(amg.AmgError) as e:
        amg.AMG(*args, coarse_enough=100, allocator=fa.struct)
    assert e.value.status == amg.AMG_ERR_CUDA and "allocator" in str(e.value)
    assert fa.calls == k and not fa.live
    assert _allocated() == base
    # the library keeps working afterwards
    u, it, res, st = amg.AMG(*args, coarse_enough=100).solve(torch.from_numpy(p.f).cuda())
    assert st == amg.AMG_OK and res <= 1e-8


@pytest.mark.parametrize("k", [1, 30, 90])
def test_failing_allocator_in_batch_setup_leaks_nothing(k):
    """The batch sets its instances up on several host threads, each calling
    the allocator; once one call fails, every instance's memory and the
    batch's own go back through the allocator."""
    mats, Bs = [], []
    for shape in ((6, 5, 7), (5, 5, 5), (7, 6, 5), (4, 6, 5), (6, 6, 6)):
        p = q.make_problem(shape, body=(0, 0, -1))
        rp, cl, val, B = dev_args(p, torch)
        mats.append((rp, cl, val))
        Bs.append(B)
    base = _allocated()
    fa = _Failing(k)
    with pytest.raises(amg.AmgError) as e:
        amg.AMGBatch(mats, Bs, [1] * 5, coarse_enough=100, allocator=fa.struct)
    assert e.value.status == amg.AMG_ERR_CUDA and "allocator" in str(e.value)
    assert fa.calls >= k and not fa.live
    assert _allocated() == base


def test_allocator_without_free_is_rejected():
    p = q.cube(4)
    args = dev_args(p, torch)
    fa = _Failing(10 ** 9)
    bad = amg.Allocator(fa.struct.alloc, amg._FREE_FN(), None)
    with pytest.raises(amg.AmgError) as e:
        amg.AMG(*args, allocator=bad)
    assert e.value.status == amg.AMG_ERR_ARG and fa.calls == 0


def test_recycled_memory_gives_the_same_solves():
    """Handles built one after another on torch's caching allocator get the
    previous handles' memory back with whatever it held (the CG's first
    direction once scaled such stale memory by beta = 0, and 0 * NaN broke
    the solve down).  Every solve must equal the one on the library's own
    allocations, bit for bit."""
    import q1elasticity as qq
    dev = torch.device("cuda:0")
    specs = qq.batch_specs(64, seed=2202)[:12]
    probs = [qq.make_problem(sp["n"], nu=sp["nu"], body=sp["body"]) for sp in specs]
    # fill torch's cache with blocks that held NaN and integers
    junk = [torch.full((1 << 22,), float("nan"), dtype=torch.float64, device=dev),
            torch.arange(1 << 23, dtype=torch.int32, device=dev)]
    del junk
    for p in probs:
        args = dev_args(p, torch)
        F = torch.from_numpy(np.atleast_2d(p.f)[:2].copy()).to(dev)
        Gt = amg.AMG(*args)
        Gn = amg.AMG(*args, allocator=None)
        for j in range(F.shape[0]):
            ut, itt, rt, st = Gt.solve(F[j])
            un, itn, rn, sn = Gn.solve(F[j])
            assert st == sn == amg.AMG_OK and (itt, rt) == (itn, rn), (p.ndof, j)
            assert torch.equal(ut, un)
        del Gt, Gn
