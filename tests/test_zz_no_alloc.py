"""pdcs_spmv_noalloc, the allocation-free product y = G x, against the
solver's own product: pdcs_solve returns the slack s = G x - h of its
returned point, computed from the solver's maintained products; the
allocation-free product of that x minus h must agree with it within 1e-9
(relative to the row's magnitude), on two calls in a row.  The file is
collected last so that it also runs after every other test."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_15504_b300 as P
    return P, torch


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def test_noalloc_product_matches_the_solver_slack_on_two_calls():
    P, torch = _env()
    prob = workloads.portfolio(n=9000, k=30, n_limits=5, limit_density=0.002, seed=11)
    lens = np.diff(prob["row_ptr"])
    # rows longer than the 4096-nonzero chunk go through the scratch
    assert (lens > 4096).sum() >= 30 and (lens <= 4096).sum() > 0
    with P.Solver(prob, max_iter=96, check_freq=32, time_limit=60.0) as s:
        r = s.solve()
    x, slack, h = r["x"], r["s"], prob["h"]
    G = workloads.to_scipy(prob)
    scale = 1.0 + abs(G) @ np.abs(x) + np.abs(h)
    rp, ci, val, xd = (_dev(torch, prob["row_ptr"]), _dev(torch, prob["col_idx"]),
                       _dev(torch, prob["val"]), _dev(torch, x))
    outs = []
    for _ in range(2):
        y = torch.full((prob["m"],), float("nan"), dtype=torch.float64, device="cuda")
        P.spmv_noalloc(rp, ci, val, xd, y)
        torch.cuda.synchronize()
        outs.append(y.cpu().numpy())
    for y in outs:
        err = np.abs((y - h) - slack) / scale
        assert err.max() <= 1e-9, err.max()
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_product_rejects_what_its_scratch_cannot_hold():
    P, torch = _env()
    # 4097 rows of 4097 nonzeros: one long row more than the scratch holds
    rows, width, n = 4097, 4097, 5000
    row_ptr = np.arange(rows + 1, dtype=np.int64) * width
    col_idx = np.tile(np.arange(width, dtype=np.int32), rows)
    val = np.ones(rows * width)
    y = torch.full((rows,), 7.0, dtype=torch.float64, device="cuda")
    assert P.spmv_noalloc_status() == 0  # no earlier call was rejected
    P.spmv_noalloc(_dev(torch, row_ptr), _dev(torch, col_idx), _dev(torch, val),
                   torch.ones(n, dtype=torch.float64, device="cuda"), y)
    # rejected on the device: counted once, nothing written, the count reset
    assert P.spmv_noalloc_status() == 1
    assert P.spmv_noalloc_status() == 0
    assert bool((y == 7.0).all())
    # one long row fewer fits, and the next call computes
    P.spmv_noalloc(_dev(torch, row_ptr[:rows]), _dev(torch, col_idx[:(rows - 1) * width]),
                   _dev(torch, val[:(rows - 1) * width]),
                   torch.ones(n, dtype=torch.float64, device="cuda"), y[:rows - 1])
    assert P.spmv_noalloc_status() == 0
    assert bool((y[:rows - 1] == float(width)).all()) and float(y[-1]) == 7.0
    # host arrays are rejected (staging copies would allocate)
    yh = np.full(2, 7.0)
    rc = P.lib().pdcs_spmv_noalloc(2, 2, row_ptr[:3].ctypes.data, col_idx.ctypes.data,
                                   val.ctypes.data, val.ctypes.data, yh.ctypes.data, None)
    assert rc == -1 and b"device memory" in P.lib().pdcs_last_error()
    assert (yh == 7.0).all()


def test_noalloc_product_small_matrix_by_definition():
    """A small matrix with empty, short and long rows against SciPy."""
    P, torch = _env()
    rng = np.random.default_rng(3)
    n = 20000
    lens = np.array([0, 1, 5, 4096, 4097, 9000, 0, 33, 12288, 2])
    cols = [np.sort(rng.choice(n, size=k, replace=False)) for k in lens]
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col_idx = np.concatenate(cols).astype(np.int32)
    val = rng.standard_normal(len(col_idx))
    x = rng.standard_normal(n)
    import scipy.sparse as sp
    ref = sp.csr_matrix((val, col_idx, row_ptr), shape=(len(lens), n)) @ x
    y = torch.empty(len(lens), dtype=torch.float64, device="cuda")
    P.spmv_noalloc(_dev(torch, row_ptr), _dev(torch, col_idx), _dev(torch, val), _dev(torch, x), y)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    scale = 1.0 + sp.csr_matrix((np.abs(val), col_idx, row_ptr), shape=(len(lens), n)) @ np.abs(x)
    assert np.max(np.abs(got - ref) / scale) <= 1e-13


def test_noalloc_product_is_captured_into_a_graph_and_replayed():
    """The call never synchronises, so after a first plain call on the device
    it can be captured: the replayed graph recomputes y from the current x."""
    P, torch = _env()
    rp = torch.tensor([0, 1, 3, 3], dtype=torch.int64, device="cuda")
    ci = torch.tensor([0, 0, 1], dtype=torch.int32, device="cuda")
    val = torch.tensor([2.0, 3.0, -1.0], dtype=torch.float64, device="cuda")
    x = torch.tensor([1.0, 1.0], dtype=torch.float64, device="cuda")
    y = torch.full((3,), 9.0, dtype=torch.float64, device="cuda")
    P.spmv_noalloc(rp, ci, val, x, y)  # the first call on the device, outside capture
    torch.cuda.synchronize()
    assert y.tolist() == [2.0, 2.0, 0.0]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            P.spmv_noalloc(rp, ci, val, x, y, stream=s)
        finally:
            g.capture_end()
    torch.cuda.current_stream().wait_stream(s)
    x.copy_(torch.tensor([0.5, -2.0], dtype=torch.float64))
    g.replay()
    torch.cuda.synchronize()
    assert y.tolist() == [1.0, 3.5, 0.0]
    # the status query synchronises, so it refuses a capturing stream
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g2.capture_begin()
        try:
            out = P.ctypes.c_int64(5)
            rc = P.lib().pdcs_spmv_noalloc_status(P.ctypes.c_void_p(s.cuda_stream),
                                                  P.ctypes.byref(out))
            y.add_(1.0)
        finally:
            g2.capture_end()
    assert rc == -1 and b"captured" in P.lib().pdcs_last_error() and out.value == 0
    g2.replay()
    torch.cuda.synchronize()
    assert y.tolist() == [2.0, 4.5, 1.0]
    assert P.spmv_noalloc_status() == 0
