"""GPU parity: Paradeisos rank/unrank and per-row index/sign lists vs the oracle, bit-exact."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle.basis import Basis, count_below, spin_list, string_at
from oracle.hamiltonian import Model, row
from tests.gpu_util import from_dev_u64, handle_for, need_gpu, to_dev_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    need_gpu()
    import paper_1707_03974_gb300 as pd
    return pd


@pytest.mark.parametrize("L", list(range(1, 21)))
def test_rank_unrank_every_spin_string(pd, L):
    """Per-spin sectors (N_dn = 0, so the combined index is the spin-up index): all n, all strings."""
    for n in range(L + 1):
        lst = spin_list(L, n)
        h = pd.Handle(L, [], [], 0.0, n, 0)
        states = to_dev_u64(lst.astype(np.uint64) << np.uint64(L))
        idx = from_dev_u64(pd.paradeisos_rank(h, states))
        assert np.array_equal(idx, np.arange(len(lst), dtype=np.uint64)), (L, n)
        back = from_dev_u64(pd.paradeisos_unrank(h, to_dev_u64(np.arange(len(lst)))))
        assert np.array_equal(back >> np.uint64(L), lst), (L, n)
        assert pd.hubbard_last_error(h) == "HB_OK"
        h.close()


@pytest.mark.parametrize("L", [24, 27, 30, 32])
def test_rank_unrank_sampled_large_L(pd, L):
    rng = np.random.default_rng(L)
    for n in (1, L // 3, L // 2, L - 1):
        D = math.comb(L, n)
        p = np.unique(np.concatenate([[0, D - 1], rng.integers(0, D, 300)]))
        strs = np.array([string_at(int(q), L, n) for q in p], dtype=np.uint64)
        assert all(count_below(int(s), L, n) == int(q) for s, q in zip(strs[:20], p[:20]))
        h = pd.Handle(L, [], [], 0.0, 0, n)  # spin-down sector: combined index = dn index
        idx = from_dev_u64(pd.paradeisos_rank(h, to_dev_u64(strs)))
        assert np.array_equal(idx, p.astype(np.uint64))
        back = from_dev_u64(pd.paradeisos_unrank(h, to_dev_u64(p)))
        assert np.array_equal(back, strs)
        assert pd.hubbard_last_error(h) == "HB_OK"
        h.close()


@pytest.mark.parametrize("L,nu,nd", [(4, 2, 3), (6, 3, 3), (8, 4, 4), (9, 2, 7), (10, 5, 4), (12, 6, 6)])
def test_combined_rank_unrank_exhaustive(pd, L, nu, nd):
    b = Basis(L, nu, nd)
    h = pd.Handle(L, [], [], 0.0, nu, nd)
    idx = from_dev_u64(pd.paradeisos_rank(h, to_dev_u64(b.combined)))
    assert np.array_equal(idx, np.arange(b.D, dtype=np.uint64))
    back = from_dev_u64(pd.paradeisos_unrank(h, to_dev_u64(np.arange(b.D))))
    assert np.array_equal(back, b.combined)
    h.close()


def test_rank_flags_invalid_strings(pd):
    L, nu, nd = 8, 3, 2
    h = pd.Handle(L, [], [], 0.0, nu, nd)
    good = (0b00010101 << L) | 0b00000011
    bad = [(0b00010111 << L) | 0b11, (0b10101 << L) | 0b111, (1 << (2 * L)) | good, 0]
    out = from_dev_u64(pd.paradeisos_rank(h, to_dev_u64([good] + bad)))
    assert out[0] != np.uint64(2 ** 64 - 1)
    assert np.all(out[1:] == np.uint64(2 ** 64 - 1))
    assert pd.hubbard_last_error(h) == "HB_ERR_INVALID_STATE"
    assert pd.hubbard_last_error(h) == "HB_OK"  # cleared
    D = math.comb(8, 3) * math.comb(8, 2)
    out = from_dev_u64(pd.paradeisos_unrank(h, to_dev_u64([0, D - 1, D, 2 ** 63])))
    assert out[0] != np.uint64(2 ** 64 - 1) and out[1] != np.uint64(2 ** 64 - 1)
    assert np.all(out[2:] == np.uint64(2 ** 64 - 1))
    assert pd.hubbard_last_error(h) == "HB_ERR_OUT_OF_RANGE"
    h.close()


def test_empty_batches(pd):
    import torch
    h = pd.Handle(6, [], [], 0.0, 3, 3)
    e = torch.empty(0, dtype=torch.int64, device="cuda")
    assert pd.paradeisos_rank(h, e).numel() == 0
    assert pd.paradeisos_unrank(h, e).numel() == 0
    h.close()


def compare_rows(pd, cl, U, nu, nd, rows, basis=None):
    b = basis if basis is not None else Basis(cl.L, nu, nd)
    m = Model.from_cluster(cl, U, nu, nd)
    h = handle_for(cl, U, nu, nd)
    rows = np.asarray(rows, dtype=np.int64)
    # contiguous runs keep the export calls few
    for r in rows:
        cols, vals, counts = pd.hubbard_row_entries(h, int(r), 1)
        n = int(counts[0])
        gc = cols[0, :n].cpu().numpy()
        gv = vals[0, :n].cpu().numpy()
        oc, ov = row(m, b, int(r))
        assert np.array_equal(gc, oc), (cl.name, r)
        assert np.array_equal(gv, ov), (cl.name, r)
    assert pd.hubbard_last_error(h) == "HB_OK"
    h.close()


def test_row_lists_ring8_all_rows(pd):
    cl = wl.ring(8)
    b = Basis(8, 4, 4)
    m = Model.from_cluster(cl, 4.0, 4, 4)
    h = handle_for(cl, 4.0, 4, 4)
    cols, vals, counts = pd.hubbard_row_entries(h, 0, b.D)
    cols, vals, counts = cols.cpu().numpy(), vals.cpu().numpy(), counts.cpu().numpy()
    for r in range(b.D):
        oc, ov = row(m, b, r)
        assert counts[r] == len(oc)
        assert np.array_equal(cols[r, :counts[r]], oc)
        assert np.array_equal(vals[r, :counts[r]], ov)
    h.close()


def test_row_of_paper_hop_example(pd):
    """Row of 0101 x 1011 on the 4-site loop: spin-up entries at 9, 1, 13 (-t) and 21 (+t)."""
    cl = wl.ring(4, t=1.0)
    h = handle_for(cl, 0.0, 2, 3)
    cols, vals, counts = pd.hubbard_row_entries(h, 5, 1)
    got = dict(zip(cols[0, :int(counts[0])].cpu().numpy().tolist(), vals[0, :int(counts[0])].cpu().numpy().tolist()))
    for c, v in {9: -1.0, 1: -1.0, 13: -1.0, 21: 1.0}.items():
        assert got[c] == v
    h.close()


@pytest.mark.parametrize("cl,nu,nd,U", [(wl.rect_periodic(4, 3), 5, 3, 7.5), (wl.ring(12), 6, 4, 2.0),
                                        (wl.rect_periodic(3, 3, 1.0, -0.3), 4, 5, 8.0)])
def test_row_lists_sampled(pd, cl, nu, nd, U):
    b = Basis(cl.L, nu, nd)
    rng = np.random.default_rng(1)
    compare_rows(pd, cl, U, nu, nd, np.unique(np.concatenate([[0, b.D - 1], rng.integers(0, b.D, 60)])), b)


def test_row_lists_square4x4_full_size_sampled(pd):
    """The 4x4 t-t' cluster at half filling (D = 165,636,900): sampled rows, bit-exact."""
    cl = wl.square_periodic(4, 1.0, -0.3)
    b = Basis(16, 8, 8)
    rng = np.random.default_rng(2)
    compare_rows(pd, cl, 8.0, 8, 8, np.unique(np.concatenate([[0, b.D - 1], rng.integers(0, b.D, 40)])), b)


def test_row_export_overflow_flag(pd):
    cl = wl.ring(8)
    h = handle_for(cl, 1.0, 4, 4)
    cols, vals, counts = pd.hubbard_row_entries(h, 0, 4, max_entries=2)
    assert np.all(counts.cpu().numpy().view(np.uint32) == 0xFFFFFFFF)
    assert pd.hubbard_last_error(h) == "HB_ERR_INVALID_ARG"
    h.close()
