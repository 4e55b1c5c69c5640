"""One binary64 problem split by block rows over two ranks (section 3.1), run as two
shards on the one GPU of this machine: each shard's local encode, ABFT product, verify and
share of a block rebuild go through the C ABI (abft_block_partial / abft_block_restore);
the two reductions that cross ranks (the grid's block checksum S_A into the rank that
holds the checksum rows, the shares of a lost block into its rank, section 3.3) are done
here by adding the shards' device buffers, which is what the NCCL reduce does between
GPUs.  The shards' kernels never wait on one another.

Checked against the oracle on the whole problem: the located faults, and the rebuilt
block within 1e-12 relative Frobenius of the oracle's rebuild and of the values before
the erasure."""
import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import abft, multigpu as mg, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_3121_gb300 import build
    build.build()
    return abft.load()


def rel_fro(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("world,lost", [(2, (1, 2)), (2, (4, 0)), (3, (5, 3))])
def test_split_grid_rebuild_and_local_correction(world, lost):
    p, q, bs, bc, k, vb = 6, 4, 64, 64, 320, 32
    m, n = p * bs, q * bc
    A = wl.operand((m, k), "normal", 17, 1)
    B = wl.operand((k, n), "normal", 17, 2)
    dev = torch.device("cuda")
    grid = mg.BlockRowGrid(p, world)
    shards = [mg.GridShard(grid, r, m, n, k, vb, vb, q, dev) for r in range(world)]
    Bt = torch.from_numpy(B).to(dev)
    Cs = []
    for sh in shards:
        A_loc = torch.from_numpy(np.ascontiguousarray(A[sh.rows.start * bs:sh.rows.stop * bs]))
        sh.encode(A_loc.to(dev), Bt, reduce=lambda t, dst: None)  # reduced below
        sh.A_loc = A_loc.to(dev)
    # the encode's reduction: every shard's local block sum into the owner's S_A rows
    owner = shards[grid.owner]
    torch.cuda.synchronize()
    total = sum(sh.s_rows().clone() for sh in shards)
    owner.s_rows().copy_(total)
    for sh in shards:
        C = torch.empty((sh.m, n), dtype=torch.float64, device=dev)
        sh.gemm(sh.A_loc, Bt, C)
        Cs.append(C)
    torch.cuda.synchronize()
    Cref = oracle.gemm(A, B)
    # a fault in one element of every shard (graded exponent flips), and the lost block
    bi, bj = lost
    flips = {}
    for r, sh in enumerate(shards):
        I = next(I for I in sh.rows if I != bi)
        i, j = (I - sh.rows.start) * bs + 5 + r, (bj + 1) % q * bc + 7
        flips[r] = (i, j)
        abft.abft_inject_bitflips(sh.desc, sh.C, [(i, j, 62)])
    r_bi = grid.rank_of(bi)
    lb = grid.local(bi)
    before = Cs[r_bi][lb * bs:(lb + 1) * bs, bj * bc:(bj + 1) * bc].cpu().numpy().copy()
    abft.abft_erase_block(shards[r_bi].desc, shards[r_bi].C, lb, bj)
    for r, sh in enumerate(shards):
        st, rep, nrep = sh.verify(erased=[lost])
        assert st == abft.OK, rep
        assert [(e["row"], e["col"]) for e in rep] == [flips[r]]
    # the rebuild: every shard's share, reduced into the rank of block row bi
    for r, sh in enumerate(shards):
        sh.share(grid.local(bi) if r == r_bi else -1, bj, r == grid.owner, sh.buf)
    torch.cuda.synchronize()
    shards[r_bi].buf.copy_(sum(sh.buf for sh in shards))
    st, ent = shards[r_bi].restore(lb, bj, shards[r_bi].buf)
    assert st == abft.OK and ent["kind"] == abft.KIND_BLOCK_RECOVERED
    got = Cs[r_bi][lb * bs:(lb + 1) * bs, bj * bc:(bj + 1) * bc].cpu().numpy()
    assert rel_fro(got, before) <= 1e-12
    # the oracle's rebuild of the whole problem from its own block checksum
    enc = oracle.Encoded(A, B, vb, vb, p, q)
    Ce = Cref.copy()
    Ce[bi * bs:(bi + 1) * bs, bj * bc:(bj + 1) * bc] = np.nan
    ost, Cr, nfl = enc.recover_block(Ce, bi, bj)
    assert ost == oracle.ST_OK and nfl == 0
    ref_blk = Cr[bi * bs:(bi + 1) * bs, bj * bc:(bj + 1) * bc]
    assert rel_fro(got, ref_blk) <= 1e-12
    # and the whole split product against the oracle's
    full = np.concatenate([C.cpu().numpy() for C in Cs])
    assert rel_fro(full, Cref) <= 1e-12


def test_block_share_and_restore_validation():
    d = abft.make_desc(128, 128, 64, "f64", 64, 64, 2, 2)
    C = torch.zeros((128, 128), dtype=torch.float64, device="cuda")
    ws = torch.zeros(abft.abft_workspace_bytes(d), dtype=torch.uint8, device="cuda")
    out = torch.empty((64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(abft.AbftError) as e:
        abft.abft_block_partial(d, C, ws, 2, 0, 0, out)
    assert e.value.status == abft.ERR_INVALID
    with pytest.raises(abft.AbftError) as e:
        abft.abft_block_partial(d, C, ws, -1, 2, 0, out)
    assert e.value.status == abft.ERR_INVALID
    nogrid = abft.make_desc(128, 128, 64, "f64", 64, 64)
    with pytest.raises(abft.AbftError) as e:
        abft.abft_block_restore(nogrid, C, ws, 0, 0, out)
    assert e.value.status == abft.ERR_INVALID
