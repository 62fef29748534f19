"""Slab decomposition (Sec. 5.1) host logic: the partition, the face layouts, the
blocks' boundary conditions and the halo exchange over gloo ranks (CPU).

The exchange is run as real torch.distributed ranks (gloo, 127.0.0.1): each rank
holds its block of a seeded whole-grid field and, after the exchange, must hold
as ghosts exactly the whole grid's cells behind each of its interface faces.
"""
import os
import socket

import numpy as np
import pytest

from paper_2112_05051_gb300 import decomp, synth

torch = pytest.importorskip("torch")


def test_partition_covers_the_grid_once_with_symmetric_neighbours():
    grid = synth.Grid(23, 17, 5)
    for px, py in ((1, 1), (2, 1), (1, 3), (3, 2), (4, 4), (23, 1)):
        blocks = decomp.partition(grid, px, py)
        assert len(blocks) == px * py and [b.rank for b in blocks] == list(range(px * py))
        owner = -np.ones((grid.ny, grid.nx), dtype=int)
        for b in blocks:
            assert np.all(owner[b.j0:b.j1, b.i0:b.i1] == -1)
            owner[b.j0:b.j1, b.i0:b.i1] = b.rank
            assert b.nbr[4] == b.nbr[5] == -1  # whole columns: no z interfaces
            for f in range(4):
                r = b.nbr[f]
                if r >= 0:
                    assert blocks[r].nbr[f ^ 1] == b.rank  # the neighbour sees b behind its opposite face
                    if f < 2:  # x neighbours share the j range, y neighbours the i range
                        assert (blocks[r].j0, blocks[r].j1) == (b.j0, b.j1)
                        assert (blocks[r].i1 if f == 0 else blocks[r].i0) == (b.i0 if f == 0 else b.i1)
                    else:
                        assert (blocks[r].i0, blocks[r].i1) == (b.i0, b.i1)
                else:
                    edge = (b.i0 == 0, b.i1 == grid.nx, b.j0 == 0, b.j1 == grid.ny)[f]
                    assert edge
        assert np.all(owner >= 0)
        widths = sorted({b.i1 - b.i0 for b in blocks})
        assert widths[-1] - widths[0] <= 1  # nearly equal
    with pytest.raises(ValueError):
        decomp.partition(grid, 24, 1)


def test_sub_grid_keeps_the_spacing_bit_for_bit():
    # the library derives h = L / (n + 1); a block's h must be the whole grid's exactly,
    # or every flux of the block rounds differently
    rng = np.random.default_rng(1)
    for _ in range(200):
        grid = synth.Grid(int(rng.integers(3, 300)), int(rng.integers(3, 300)), 5, float(rng.uniform(0.1, 1e3)),
                          float(rng.uniform(0.1, 1e3)), 1.5)
        for b in decomp.partition(grid, min(3, grid.nx), min(2, grid.ny)):
            sg = decomp.sub_grid(grid, b)
            assert (sg.nx, sg.ny, sg.nz) == (b.i1 - b.i0, b.j1 - b.j0, grid.nz)
            assert sg.h == grid.h  # carried explicitly: l / (n + 1) of the block's box need not give it


def _pack(l3, f):
    """Cells next to face f of a block array (nz, ny, nx), in the face layout."""
    return [l3[:, :, 0], l3[:, :, -1], l3[:, 0, :], l3[:, -1, :], l3[0], l3[-1]][f].reshape(-1)


def test_face_layout_and_ghost_planes_match_the_index_formulas():
    grid = synth.Grid(9, 7, 4)
    a3 = np.arange(grid.n, dtype=np.float64).reshape(grid.shape)  # value = global cell index
    blocks = decomp.partition(grid, 3, 2)
    for b in blocks:
        nx, ny = b.i1 - b.i0, b.j1 - b.j0
        l3 = decomp.cell_block(a3, b)
        for f in range(6):
            face = _pack(l3, f)
            assert len(face) == decomp.face_cells(decomp.sub_grid(grid, b), f)
            for t, v in enumerate(face):  # the documented index of each face layout
                if f < 2:
                    j, k, i = t % ny, t // ny, (0 if f == 0 else nx - 1)
                elif f < 4:
                    i, k, j = t % nx, t // nx, (0 if f == 2 else ny - 1)
                else:
                    i, j, k = t % nx, t // nx, (0 if f == 4 else grid.nz - 1)
                assert v == (b.i0 + i) + grid.nx * ((b.j0 + j) + grid.ny * k)
            r = b.nbr[f]
            if r >= 0:  # the ghosts of face f are the cells the neighbour packs on its face f ^ 1
                np.testing.assert_array_equal(decomp.ghost_plane(a3, b, f).reshape(-1),
                                              _pack(decomp.cell_block(a3, blocks[r]), f ^ 1))


def test_block_bc_slices_outer_fields_and_carries_ghost_ks():
    from paper_2112_05051_gb300 import richards as rb
    grid = synth.Grid(12, 10, 6)
    bc = synth.paper_infiltration_bc(grid, -30.0)  # per-cell values on the top face
    ks = synth.ks_field(grid, 4, 1.0)
    k3 = ks.reshape(grid.shape)
    top = np.asarray(bc.field(5)).reshape(grid.ny, grid.nx)
    for b in decomp.partition(grid, 2, 2):
        bb = decomp.block_bc(grid, bc, b, ks)
        for f in range(6):
            if b.nbr[f] >= 0:
                assert bb.kind[f] == rb.BC_INTERFACE
                np.testing.assert_array_equal(bb.ghost_ks_field(f), decomp.ghost_plane(k3, b, f).reshape(-1))
                assert len(bb.field(f)) == decomp.face_cells(decomp.sub_grid(grid, b), f)
            else:
                assert bb.kind[f] == bc.kind[f] and bb.value[f] == bc.value[f] and bb.ghost_ks_field(f) is None
        np.testing.assert_array_equal(bb.field(5), top[b.j0:b.j1, b.i0:b.i1].reshape(-1))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange_rank(rank, world, port, px, py, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid = synth.Grid(11, 9, 4)
        a3 = np.random.default_rng(3).standard_normal(grid.shape)
        blocks = decomp.partition(grid, px, py)
        b = blocks[rank]
        l3 = torch.tensor(np.ascontiguousarray(decomp.cell_block(a3, b)))
        halo = decomp.Halo(blocks, rank)
        got = {}
        sg = decomp.sub_grid(grid, b)
        buffers = {f: (torch.empty(decomp.face_cells(sg, f), dtype=torch.float64),
                       torch.empty(decomp.face_cells(sg, f), dtype=torch.float64))
                   for f in range(6) if b.nbr[f] >= 0}
        pack = lambda f, out: out.copy_(_pack(l3, f))
        apply = lambda f, ghosts: got.__setitem__(f, ghosts.clone().numpy())
        for _ in range(2):  # twice: buffers are reused
            halo.exchange(dist, pack, apply, buffers)
        ok = all(np.array_equal(got[f], decomp.ghost_plane(a3, b, f).reshape(-1)) for f in got)
        ok = ok and set(got) == {f for f in range(6) if b.nbr[f] >= 0}
        open(os.path.join(out_dir, "rank%d" % rank), "w").write("ok" if ok else "bad")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 2), (3, 1)])
def test_halo_exchange_on_gloo_ranks(px, py, tmp_path):
    import torch.multiprocessing as mp
    world = px * py
    mp.spawn(_exchange_rank, args=(world, _free_port(), px, py, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        assert (tmp_path / ("rank%d" % r)).read_text() == "ok"


def _comm_rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = decomp.DistComm(dist, None, "cpu")
        vals = [1e16, 1.0, -1e16, 3.5][:world]  # a plain sum depends on the order of the terms
        s = comm.sum([vals[rank]])
        m = comm.max([vals[rank]])
        ok = s == sum(vals) == 4.5 and m == max(vals)  # every rank's value, compensated, in rank order
        open(os.path.join(out_dir, "rank%d" % rank), "w").write("%r %r %s" % (s, m, ok))
    finally:
        dist.destroy_process_group()


def test_dist_comm_sums_in_rank_order_on_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 4
    mp.spawn(_comm_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    outs = [(tmp_path / ("rank%d" % r)).read_text() for r in range(world)]
    assert all(o.endswith("True") for o in outs) and len(set(outs)) == 1  # the same sum on every rank
