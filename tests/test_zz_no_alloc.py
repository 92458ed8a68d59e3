"""The allocation-free solve (csp_solve_static) against the allocating one (csp_solve).

Some callers cannot allocate device memory: code that runs inside a framework or runtime
that owns every device allocation, or under a memory cap.  csp_solve_static keeps the
solver's scratch in a static device array of the library instead.  Here it is called
through the C ABI, two calls in a row (and then on other instances, among them a 3-D
lattice with 16-bit weights, whose 32-byte edge records the static layout sizes apart),
and each result must equal csp_solve's exactly: every output is an integer, so the
tolerance is zero, as in the other parity tests.

The file's name makes pytest collect it last, so that a run which stops at the first
failure has run every other test before this one; it does not depend on them and passes
alone in a fresh process as well.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _devices(torch, inst):
    cuda = torch.device("cuda")
    return (torch.from_numpy(inst.f1).to(cuda), torch.from_numpy(inst.f2).to(cuda),
            torch.from_numpy(inst.A).to(cuda), torch.from_numpy(inst.B).to(cuda))


def test_static_solve_equals_csp_solve_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    from paper_1511_06441_gb300 import build, csp, synth
    build.build()
    cube = synth.workload_cube(40, 500)
    grid = synth.workload_64x64()
    ext16 = [24, 24, 24]  # 16-bit weights with d = 3: 32-byte edge records
    g1, g2 = synth.uniform_weights(ext16, 1, 300, 17, dtype=np.uint16)
    wide = synth.Instance(ext16, g1, g2, synth.face(ext16, 0, 0), synth.face(ext16, 0, 23), 3000, "cube24_u16")
    cases = [(cube, 500), (cube, 500), (grid, 300), (wide, 3000), (wide, 3000), (cube, 350)]
    want = {}
    for inst, M in cases:
        if (inst.name, M) not in want:
            lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
            want[(inst.name, M)] = lat.solve(inst.A, inst.B, M)
            lat.close()
    rec = torch.full((16,), -7, dtype=torch.int64, device="cuda")
    for inst, M in cases:
        f1, f2, A, B = _devices(torch, inst)
        torch.cuda.synchronize()
        csp.solve_static(inst.extents, f1, f2, A, B, M, rec)
        torch.cuda.synchronize()
        got = csp.result_from_record(rec.cpu().numpy())
        w = want[(inst.name, M)]
        assert got.status == csp.OK
        assert got.answer() == w.answer()
        assert (got.cycles, got.updates, got.launched, got.arrivals, got.improved) == \
               (w.cycles, w.updates, w.launched, w.arrivals, w.improved)


def test_static_solve_rejects_oversized_lattices_and_bad_inputs():
    torch = pytest.importorskip("torch")
    from paper_1511_06441_gb300 import build, csp, synth
    build.build()
    ext = [2048, 2048]  # 4.2M vertices: the vertex arrays alone exceed the static array
    f1 = torch.zeros((2, 2048 * 2048), dtype=torch.uint8, device="cuda")
    A = torch.tensor([0], dtype=torch.int64, device="cuda")
    B = torch.tensor([5], dtype=torch.int64, device="cuda")
    rec = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(csp.CspError) as e:
        csp.solve_static(ext, f1, f1, A, B, 100, rec)
    assert e.value.status == csp.ERR_INVALID and "static workspace" in str(e.value)
    # overlapping A and B are reported in the record, as for csp_solve_async
    inst = synth.workload_cube(16, 200)
    f1d, f2d, Ad, _ = _devices(torch, inst)
    csp.solve_static(inst.extents, f1d, f2d, Ad, Ad, 200, rec)
    torch.cuda.synchronize()
    assert int(rec[0].item()) == csp.ERR_INVALID
    # nonzero upper-face travel times are refused (no private copy to zero them in)
    bad = f1d.clone()
    bad[0, 15] = 3  # vertex (15, 0, 0) lies on the upper face of dimension 0
    csp.solve_static(inst.extents, bad, f2d, Ad, torch.from_numpy(inst.B).cuda(), 200, rec)
    torch.cuda.synchronize()
    assert int(rec[0].item()) == csp.ERR_INVALID
