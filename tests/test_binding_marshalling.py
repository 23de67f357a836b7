"""The Python binding's argument marshalling, on the CPU, against a stand-in
for the library that records every call: each entry point hands the C ABI
the arrays' own pointers and sizes, and an array whose element type or
length differs from what the library reads through it is rejected before
any library call (the library would read or write past its end)."""
import ctypes as C

import numpy as np
import pytest

from paper_2502_17632_gb300 import gift

N, S = 10, 3


class FakeLib:
    def __init__(self, cells=N):
        self.calls = []
        self.cells = cells

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, args))
            if name == "gift_graph_info":
                args[1]._obj.num_cells = self.cells
            return gift.GIFT_OK
        return call

    def names(self):
        return [c[0] for c in self.calls]


@pytest.fixture
def lib(monkeypatch):
    fake = FakeLib()
    monkeypatch.setattr(gift, "load", lambda *a, **k: fake)
    return fake


def sig(n=N, s=S, dtype=np.float32):
    return np.zeros((n, s, 2), dtype=dtype)


def netlist():
    net_ptr = np.array([0, 3, 5, 9], dtype=np.int64)
    pin_cell = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8], dtype=np.int32)
    return net_ptr, pin_cell, np.zeros(N, np.uint8)


def test_filter_passes_the_arrays_own_pointers(lib):
    g, out = sig(), sig()
    gift.gift_filter(None, 1, g, out)
    name, args = lib.calls[-1]
    assert name == "gift_filter"
    assert args[3] == g.ctypes.data and args[4] == S and args[5] == out.ctypes.data
    assert args[6] == gift.GIFT_MEM_HOST


@pytest.mark.parametrize("bad", ["dtype", "short", "strided"])
def test_filter_rejects_bad_signals(lib, bad):
    g = {"dtype": sig(dtype=np.float64), "short": sig(n=N - 1), "strided": sig(s=2 * S)[:, ::2]}[bad]
    with pytest.raises((TypeError, ValueError)):
        gift.gift_filter(None, 1, g, sig(), num_signals=S)
    with pytest.raises((TypeError, ValueError)):
        gift.gift_filter(None, 1, sig(), g, num_signals=S)
    assert "gift_filter" not in lib.names()


def test_filter_signal_count_is_checked_against_the_arrays(lib):
    with pytest.raises(ValueError):
        gift.gift_filter(None, 1, sig(), sig(), num_signals=S + 1)
    gift.gift_filter(None, 1, sig(), sig(), num_signals=0)  # the library rejects 0 itself
    assert lib.names().count("gift_filter") == 1


def test_build_graph_types_and_lengths(lib):
    net_ptr, pin_cell, fx = netlist()
    gift.gift_build_graph(None, N, net_ptr, pin_cell, fx)
    name, args = lib.calls[-1]
    nl = args[1]._obj
    assert name == "gift_build_graph"
    assert (nl.num_cells, nl.num_nets, nl.net_ptr, nl.pin_cell, nl.is_fixed) == \
        (N, 3, net_ptr.ctypes.data, pin_cell.ctypes.data, fx.ctypes.data)
    gift.gift_build_graph(None, N, net_ptr, pin_cell, fx.astype(bool))  # one byte per cell as well
    for bad in [dict(net_ptr=net_ptr.astype(np.int32)), dict(pin_cell=pin_cell.astype(np.int64)),
                dict(pin_cell=pin_cell[:-1]), dict(is_fixed=fx[:-1]), dict(is_fixed=fx.astype(np.int32)),
                dict(net_ptr=net_ptr[:0])]:
        kw = dict(net_ptr=net_ptr, pin_cell=pin_cell, is_fixed=fx)
        kw.update(bad)
        with pytest.raises((TypeError, ValueError)):
            gift.gift_build_graph(None, N, kw["net_ptr"], kw["pin_cell"], kw["is_fixed"])
    assert lib.names().count("gift_build_graph") == 2


def test_torch_tensors_are_checked_too(lib):
    torch = pytest.importorskip("torch")
    net_ptr, pin_cell, fx = netlist()
    with pytest.raises(TypeError):
        gift.gift_build_graph(None, N, torch.from_numpy(net_ptr.astype(np.int32)), torch.from_numpy(pin_cell),
                              None)
    with pytest.raises(TypeError):
        gift.gift_hpwl(None, 1, torch.zeros((N, S, 2), dtype=torch.float64))
    gift.gift_hpwl(None, 1, torch.zeros((N, S, 2), dtype=torch.float32))
    assert lib.names().count("gift_hpwl") == 1


def test_hpwl_tikhonov_eigen_density(lib):
    gift.gift_hpwl(None, 1, sig())
    with pytest.raises(ValueError):
        gift.gift_hpwl(None, 1, sig(n=N - 1))
    gift.gift_tikhonov(None, 1, sig(), sig())
    with pytest.raises(TypeError):
        gift.gift_tikhonov(None, 1, sig(), sig(dtype=np.float16))
    out, _ = gift.gift_eigen_placement(None, 1)
    assert out.shape == (N, 2) and out.dtype == np.float64
    with pytest.raises(TypeError):
        gift.gift_eigen_placement(None, 1, out=np.zeros((N, 2), np.float32))
    with pytest.raises(ValueError):
        gift.gift_eigen_placement(None, 1, out=np.zeros((N - 1, 2), np.float64))
    w = np.ones(N, np.float32)
    gift.gift_density(None, sig(), cell_w=w, cell_h=w)
    with pytest.raises(TypeError):
        gift.gift_density(None, sig(), cell_w=w.astype(np.float64), cell_h=w)
    with pytest.raises(ValueError):
        gift.gift_density(None, sig(), cell_w=w[:-1], cell_h=w)
    assert lib.names().count("gift_tikhonov") == 1 and lib.names().count("gift_eigen_placement") == 1
    assert lib.names().count("gift_density") == 1 and lib.names().count("gift_hpwl") == 1


def test_run_and_batches(lib):
    net_ptr, pin_cell, fx = netlist()
    gift.gift_run(None, N, net_ptr, pin_cell, fx, sig(), sig())
    with pytest.raises(TypeError):
        gift.gift_run(None, N, net_ptr, pin_cell, fx, sig(), sig(dtype=np.float64))
    with pytest.raises(ValueError):
        gift.gift_run(None, N, net_ptr, pin_cell[:-1], fx, sig(), sig())
    with pytest.raises(ValueError):
        gift.gift_run(None, N, net_ptr, pin_cell, fx, sig(), sig(n=N - 1))
    assert lib.names().count("gift_run") == 1
    gift.gift_build_batch(None, [(N, net_ptr, pin_cell, fx), (N, net_ptr, pin_cell, None)])
    with pytest.raises(ValueError):
        gift.gift_build_batch(None, [(N, net_ptr, pin_cell[:-2], fx)])
    assert lib.names().count("gift_build_batch") == 1
    lib.cells = 2 * N
    gift.gift_hpwl_batch(None, 1, sig(n=2 * N), 2)
    with pytest.raises(ValueError):
        gift.gift_hpwl_batch(None, 1, sig(n=N), 2)
    with pytest.raises(TypeError):
        gift.gift_filter_capture(None, 1, sig(n=2 * N, dtype=np.float64), sig(n=2 * N))
