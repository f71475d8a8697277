"""Parameter selection through the C ABI (snaps_select; Sec. 3.5.2, Eq. 2 and
3; Sec. 3.6.2) against the FP64 oracle, which runs one full join per grid
value: the same U^min / U^max curves and the same selected grid index per
metric, for subspaces of 2, 6 and 15 features and k grids up to 4096; and the
invalid requests it must reject."""
import numpy as np
import pytest

import oracle
import paper_2405_20176_b300 as snaps
import snaps_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = snaps.snaps_create(0)
    yield c
    snaps.snaps_destroy(c)


@pytest.mark.parametrize("n,seed", [(1500, 0), (777, 3)])
def test_select_matches_oracle(ctx, n, seed):
    x = snaps_inputs.population(n, seed)
    masks = np.array([0b11000, 0b101000110100010, (1 << 15) - 1], dtype=np.uint16)
    d = np.array([bin(int(m)).count("1") for m in masks])
    eps_min = (0.02 * np.sqrt(d)).astype(np.float32)
    eps_max = (0.12 * np.sqrt(d)).astype(np.float32)
    n_eps = 8
    k_grid = [2, 4, 8, 16, 32]
    top_n = max(1, n // 100)
    pop = snaps.snaps_index(ctx, x)
    try:
        u_eps, e_sel, u_k, k_sel = snaps.snaps_select(pop, masks, eps_min, eps_max, n_eps, k_grid, top_n)
    finally:
        snaps.snaps_release(pop)
    xn = oracle.normalise(x)
    for s, m in enumerate(masks):
        u, sel, _ = oracle.select_eps(xn, int(m), float(eps_min[s]), float(eps_max[s]), n_eps, top_n)
        np.testing.assert_allclose(u_eps[s], u, atol=1e-6, err_msg=f"eps U, mask {int(m):#x}")
        np.testing.assert_array_equal(e_sel[s], sel)
        uk, selk, _ = oracle.select_k(xn, int(m), k_grid, top_n)
        np.testing.assert_allclose(u_k[s], uk, atol=1e-6, err_msg=f"k U, mask {int(m):#x}")
        np.testing.assert_array_equal(k_sel[s], selk)


@pytest.mark.parametrize("n,seed,k_grid", [(1500, 4, [2, 8, 64, 256, 1024, 1499]),
                                           (4200, 6, [33, 1024, 4096])])
def test_select_large_k_matches_oracle(ctx, n, seed, k_grid):
    # k grids beyond 32 (the paper's reach 4096) take the CTA-per-object path
    x = snaps_inputs.population(n, seed)
    masks = np.array([0b110000, 0b111111100000000], dtype=np.uint16)[: 2 if n < 2000 else 1]
    top_n = max(1, n // 100)
    pop = snaps.snaps_index(ctx, x)
    try:
        _, _, u_k, k_sel = snaps.snaps_select(pop, masks, k_grid=k_grid, top_n=top_n)
    finally:
        snaps.snaps_release(pop)
    xn = oracle.normalise(x)
    for s, m in enumerate(masks):
        uk, selk, _ = oracle.select_k(xn, int(m), k_grid, top_n)
        np.testing.assert_allclose(u_k[s], uk, atol=1e-6, err_msg=f"k U, mask {int(m):#x}")
        np.testing.assert_array_equal(k_sel[s], selk)


def test_select_one_grid_only(ctx):
    x = snaps_inputs.population(600, 1)
    masks = np.array([0b110], dtype=np.uint16)
    pop = snaps.snaps_index(ctx, x)
    try:
        u_eps, e_sel, u_k, k_sel = snaps.snaps_select(pop, masks, k_grid=[3, 9], top_n=6)
        assert u_eps is None and e_sel is None and u_k.shape == (1, 2, 2, 2)
        u_eps, e_sel, u_k, k_sel = snaps.snaps_select(pop, masks, 0.01, 0.2, 4, top_n=6)
        assert u_k is None and u_eps.shape == (1, 2, 2, 4)
    finally:
        snaps.snaps_release(pop)


def test_select_rejects_bad_grids(ctx):
    x = snaps_inputs.population(300, 2)
    masks = np.array([0b110], dtype=np.uint16)
    pop = snaps.snaps_index(ctx, x)
    try:
        for kw in (dict(eps_min=0.2, eps_max=0.1, n_eps=4),         # empty range
                   dict(eps_min=0.1, eps_max=0.2, n_eps=1),         # one value
                   dict(eps_min=0.1, eps_max=0.2, n_eps=65),        # too many
                   dict(k_grid=[4, 2]),                             # not ascending
                   dict(k_grid=[2, 4097]),                          # beyond SNAPS_SELECT_MAX_K
                   dict(k_grid=[2, 300]),                           # beyond n - 1
                   dict(k_grid=[2, 4], top_n=0)):
            kw.setdefault("top_n", 3)
            with pytest.raises(snaps.SnapsError) as e:
                snaps.snaps_select(pop, masks, **kw)
            assert e.value.status == snaps.SNAPS_EINVAL
    finally:
        snaps.snaps_release(pop)
