"""One Taylor-Couette case split across ranks: partition and exchanges.

The paper distributes one case over the nodes of a cluster by radial slabs
and pipelines the banded radial solves through them (Sec. 3.1).  Here the
split is the transpose form: the plane phase (transforms in theta and z and
the products, independent per radial plane) runs on radial slabs, the line
phase (rows of Eqs. 6-7 and the radial solves, independent per Fourier pair)
on azimuthal columns, and two all-to-all exchanges per substep move the data
between the two partitions:

  A. before the plane phase, u, v, w of every rank's columns go to the ranks
     owning the planes (each rank receives the other ranks' columns on its
     planes);
  B. after it, the products of every rank's planes go to the ranks owning
     the columns.

The rank that owns azimuthal column 0 also advances the mean flow (U, W live
in the (0, 0) slot of u and w and travel with column 0 in exchange A; the
(0, 0) products it needs arrive in exchange B).

Every array is a tensor whose last axis holds the bytes of one complex
element as float32 words (4 for complex128 and the double-float pairs, 2 for
complex64), so the exchanges move bytes and the split reproduces the
unsplit step bit for bit.  The tensors can live on any device; the transport
is a callable taking one send tensor per destination rank and returning one
received tensor per source rank (`all_to_all` below wraps
torch.distributed.all_to_all_single; `exchange_in_process` stands in for it
when all shares live in one process).

The compute of a share is given as two callables, planes() and pairs(k);
`libtc_share` binds them to the libtc calls tc_split_planes / tc_split_pairs
of a handle whose resident arrays the tensors view.
"""
import torch


def balanced(n, parts):
    """Contiguous ranges [a, b) covering 0..n-1, sizes differing by at most 1."""
    if parts < 1 or n < parts:
        raise ValueError(f"cannot split {n} items into {parts} non-empty parts")
    base, extra = divmod(n, parts)
    out, a = [], 0
    for p in range(parts):
        b = a + base + (1 if p < extra else 0)
        out.append((a, b))
        a = b
    return out


class SplitPlan:
    """Radial slabs and azimuthal columns of each of `world` ranks."""

    def __init__(self, Nr, Ntheta, Nz, world):
        self.Nr, self.Nz, self.Nh, self.world = Nr, Nz, Ntheta // 2, world
        self.slabs = balanced(Nr, world)
        self.cols = balanced(self.Nh, world)


# ---- exchange A: u, v, w from column owners to plane owners -----------------

def pack_to_planes(plan, rank, fields):
    """fields: tensors [Nr][Nz][Nh][E]; one send tensor per destination q: the
    fields on q's planes, this rank's columns."""
    j0, j1 = plan.cols[rank]
    return [torch.stack([f[r0:r1, :, j0:j1] for f in fields]).contiguous() for (r0, r1) in plan.slabs]


def unpack_to_planes(plan, rank, fields, recvs):
    """recvs[p]: the fields on this rank's planes, columns of rank p."""
    r0, r1 = plan.slabs[rank]
    for p, blk in enumerate(recvs):
        if p == rank:
            continue
        j0, j1 = plan.cols[p]
        for i, f in enumerate(fields):
            f[r0:r1, :, j0:j1] = blk[i]


# ---- exchange B: products from plane owners to column owners ----------------

def pack_to_pairs(plan, rank, slab_prod):
    """slab_prod: [nprod][r1-r0][Nz][Nh][E] (this rank's planes); one send
    tensor per destination q: q's columns."""
    return [slab_prod[:, :, :, j0:j1].contiguous() for (j0, j1) in plan.cols]


def unpack_to_pairs(plan, rank, full_prod, recvs):
    """full_prod: [nprod][Nr][Nz][Nh][E]; recvs[p]: rank p's planes of the
    products in this rank's columns."""
    j0, j1 = plan.cols[rank]
    for p, blk in enumerate(recvs):
        r0, r1 = plan.slabs[p]
        full_prod[:, r0:r1, :, j0:j1] = blk


# ---- transports -----------------------------------------------------------

def all_to_all(sends, recv_shapes, group=None):
    """One all-to-all of torch.distributed: sends[q] goes to rank q; returns
    the tensors received from every rank, shaped recv_shapes[p] (every rank
    knows them from the common plan)."""
    import torch.distributed as dist
    flat = torch.cat([s.reshape(-1) for s in sends])
    in_splits = [s.numel() for s in sends]
    out_splits = [int(torch.Size(sh).numel()) for sh in recv_shapes]
    out = torch.empty(sum(out_splits), dtype=flat.dtype, device=flat.device)
    dist.all_to_all_single(out, flat, out_splits, in_splits, group=group)
    return [o.reshape(sh) for o, sh in zip(out.split(out_splits), recv_shapes)]


def recv_shapes_planes(plan, rank, nfields, E):
    r0, r1 = plan.slabs[rank]
    return [(nfields, r1 - r0, plan.Nz, j1 - j0, E) for (j0, j1) in plan.cols]


def recv_shapes_pairs(plan, rank, nprod, E):
    j0, j1 = plan.cols[rank]
    return [(nprod, r1 - r0, plan.Nz, j1 - j0, E) for (r0, r1) in plan.slabs]


def exchange_in_process(sends_by_rank):
    """The all-to-all among shares held by one process: recv[q][p] = send[p][q]."""
    n = len(sends_by_rank)
    return [[sends_by_rank[p][q] for p in range(n)] for q in range(n)]


# ---- one rank's share -----------------------------------------------------

class Share:
    """Arrays and compute of one rank's share of a split case.

    arrays: "u", "v", "w" [Nr][Nz][Nh][E], "prod" [nprod][Nr][Nz][Nh][E],
    "prod_slab" [nprod][r1-r0][Nz][Nh][E]; planes(): the plane phase of the
    rank's slab; pairs(k): the line phase (and mean flow) of substep k."""

    def __init__(self, plan, rank, arrays, planes, pairs):
        self.plan, self.rank, self.a = plan, rank, arrays
        self.planes, self.pairs = planes, pairs

    def fields(self):
        return [self.a["u"], self.a["v"], self.a["w"]]


def step_distributed(share, group=None):
    """One Runge-Kutta step of this rank's share, exchanging with the other
    ranks of the torch.distributed group (every rank calls it)."""
    plan, rank = share.plan, share.rank
    E = share.a["u"].shape[-1]
    nprod = share.a["prod"].shape[0]
    for k in range(3):
        recvs = all_to_all(pack_to_planes(plan, rank, share.fields()),
                           recv_shapes_planes(plan, rank, 3, E), group)
        unpack_to_planes(plan, rank, share.fields(), recvs)
        share.planes()
        recvs = all_to_all(pack_to_pairs(plan, rank, share.a["prod_slab"]),
                           recv_shapes_pairs(plan, rank, nprod, E), group)
        unpack_to_pairs(plan, rank, share.a["prod"], recvs)
        share.pairs(k)


def step_in_process(shares):
    """One Runge-Kutta step of all shares of a case held by one process, the
    exchanges done by copies (no rank waits on another)."""
    plan = shares[0].plan
    for k in range(3):
        recvs = exchange_in_process([pack_to_planes(plan, s.rank, s.fields()) for s in shares])
        for s in shares:
            unpack_to_planes(plan, s.rank, s.fields(), recvs[s.rank])
            s.planes()
        recvs = exchange_in_process([pack_to_pairs(plan, s.rank, s.a["prod_slab"]) for s in shares])
        for s in shares:
            unpack_to_pairs(plan, s.rank, s.a["prod"], recvs[s.rank])
            s.pairs(k)


# ---- the share of a libtc handle --------------------------------------------

class _CudaArray:
    """__cuda_array_interface__ of a device buffer, for a zero-copy tensor."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_tensor(ptr, shape):
    return torch.as_tensor(_CudaArray(ptr, shape), device="cuda")


def libtc_share(h, plan, rank, precision):
    """The share of rank `rank` on a libtc handle h of the whole case (any
    precision form; the handle's launch stream must be torch's current
    stream, so that the copies of the exchanges and the kernels stay in
    order)."""
    import paper_0711_1429_gb300 as tc
    (r0, r1), (j0, j1) = plan.slabs[rank], plan.cols[rank]
    tc.tc_split_set(h, r0, r1, j0, j1)
    Nr, Nz, Nh = plan.Nr, plan.Nz, plan.Nh
    Ep = 2 if precision == tc.TC_PREC_MIXED else 4
    arrays = {name: device_tensor(tc.tc_device_array(h, which), (Nr, Nz, Nh, 4))
              for name, which in (("u", tc.TC_ARRAY_U), ("v", tc.TC_ARRAY_V), ("w", tc.TC_ARRAY_W))}
    arrays["prod"] = device_tensor(tc.tc_device_array(h, tc.TC_ARRAY_PROD), (5, Nr, Nz, Nh, Ep))
    arrays["prod_slab"] = device_tensor(tc.tc_device_array(h, tc.TC_ARRAY_PROD_SLAB), (5, r1 - r0, Nz, Nh, Ep))
    return Share(plan, rank, arrays, lambda: tc.tc_split_planes(h), lambda k: tc.tc_split_pairs(h))
