"""md_nb_gradient_noalloc: the nonbonded gradient for callers that cannot
allocate device memory (for example, a host framework whose allocator owns
the GPU's memory, or a real-time loop that cannot afford the synchronisation
of cudaMalloc). The caller passes device arrays for inputs and output; the
entry point uses a static device scratch array and allocates nothing.

Checked through the C ABI against md_gradient of an FP64 context (modes 2, 3
and 4: full, short and long pair gradients), on two calls in a row each, with
the output buffer poisoned before every call; the two calls return the same
bits. With no molecule ids (no exclusions) it is checked against the FP64
oracle's brute-force pair sum.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2, skin=0.2, skin_outer=0.3)


def rel_err(g, ref):
    rms = np.sqrt((ref * ref).sum(1).mean())
    den = np.maximum(np.linalg.norm(ref, axis=1), 0.01 * rms)
    return (np.linalg.norm(g - ref, axis=1) / den).max()


@pytest.mark.parametrize("n_mol,box", [(216, 18.643), (2000, None)])
def test_noalloc_gradient_matches_context_path(n_mol, box):
    import torch

    import paper_2412_15073_gb300 as M
    from paper_2412_15073_gb300 import systems

    L = M.load_library()
    w = systems.water_box(n_mol, box=box, seed=4)
    e = M.Engine(precision=M.MD_FP64)
    e.set_system(0, w, **P)
    refs = {weight: e.gradient(2 + weight) for weight in (0, 1, 2)}
    e.close()

    dev = torch.device("cuda", 0)
    x = torch.tensor(w.x, dtype=torch.float64, device=dev).contiguous()
    q = torch.tensor(w.charge, dtype=torch.float64, device=dev)
    t = torch.tensor(w.type, dtype=torch.int32, device=dev)
    mol = torch.arange(w.n, dtype=torch.int32, device=dev) // 3
    grad = torch.empty((w.n, 3), dtype=torch.float64, device=dev)
    eps = np.ascontiguousarray(w.lj_eps, dtype=np.float64)
    sig = np.ascontiguousarray(w.lj_sigma, dtype=np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    first = {}
    for call in range(2):
        for weight in (0, 1, 2):
            grad.fill_(float("nan"))
            rc = L.md_nb_gradient_noalloc(
                ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                ctypes.c_void_p(mol.data_ptr()), w.n, w.box, eps.shape[0], M._ptr(eps), M._ptr(sig),
                P["r_cut"], P["r_split"], P["h_switch"], P["dsf_alpha"], weight,
                ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(stream))
            assert rc == 0, L.md_last_error(None).decode()
            torch.cuda.synchronize()
            g = grad.cpu().numpy()
            assert np.isfinite(g).all()
            err = rel_err(g, refs[weight])
            assert err <= 1e-12, (call, weight, err)
            if call == 0:
                first[weight] = g.copy()
            else:
                assert np.array_equal(g, first[weight]), weight     # fixed summation order


def test_noalloc_without_molecule_ids_matches_the_oracle():
    """d_mol = NULL: every pair interacts (no exclusions); 300 charged LJ
    beads at random positions (no two closer than 2.6 A) in a 22 A box,
    against the oracle's brute-force FP64 pair gradients of the same weights."""
    import torch

    import oracle
    import paper_2412_15073_gb300 as M
    from paper_2412_15073_gb300 import systems

    rng = np.random.default_rng(11)
    box, pts = 22.0, []
    while len(pts) < 300:
        c = rng.uniform(0, box, 3)
        if all(np.linalg.norm((c - p) - box * np.round((c - p) / box)) > 2.6 for p in pts):
            pts.append(c)
    q = np.where(np.arange(300) % 2 == 0, 0.5, -0.5)
    w = systems.point_charges(np.array(pts), box, q, 20.0, lj_eps=0.2, lj_sigma=3.2)
    oracle.build()
    o = oracle.Oracle(w, r_cut=9.0, r_split=5.0, h_switch=0.5, dsf_alpha=0.2, skin=0.2)
    refs = {weight: o.gradient(2 + weight)[0] for weight in (0, 1, 2)}
    L = M.load_library()
    dev = torch.device("cuda", 0)
    x = torch.tensor(w.x, dtype=torch.float64, device=dev).contiguous()
    qd = torch.tensor(w.charge, dtype=torch.float64, device=dev)
    t = torch.tensor(w.type, dtype=torch.int32, device=dev)
    grad = torch.empty((w.n, 3), dtype=torch.float64, device=dev)
    eps = np.ascontiguousarray(w.lj_eps, dtype=np.float64)
    sig = np.ascontiguousarray(w.lj_sigma, dtype=np.float64)
    for weight in (0, 1, 2):
        grad.fill_(float("nan"))
        rc = L.md_nb_gradient_noalloc(
            ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(qd.data_ptr()), ctypes.c_void_p(t.data_ptr()),
            None, w.n, w.box, 1, M._ptr(eps), M._ptr(sig), 9.0, 5.0, 0.5, 0.2, weight,
            ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, L.md_last_error(None).decode()
        torch.cuda.synchronize()
        err = rel_err(grad.cpu().numpy(), refs[weight])
        assert err <= 1e-12, (weight, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_2412_15073_gb300 as M
    L = M.load_library()
    one = np.zeros(1)
    rc = L.md_nb_gradient_noalloc(M._ptr(one), M._ptr(one), M._ptr(one), None, 200_000, 1000.0, 1,
                                  M._ptr(one), M._ptr(one), 9.0, 5.0, 0.5, 0.2, 0, M._ptr(one), None)
    assert rc == -1
    assert b"MD_NOALLOC_MAX_ATOMS" in L.md_last_error(None)
