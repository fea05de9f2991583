"""Z-slab decomposition of one 3D grid over the ranks of a process group:
the exchange steps of the equilibrium PCG (Sec. 2.3) when one grid is split
along z across devices.

Each rank holds planes [z0, z1) of every field. One PCG iteration on the
potential (K u = f, K = grad+^T g C grad+, preconditioner M^-1 = F^-1
(1 / (m1 |D|^2)) F per component) needs three exchanges:
- one-plane halos: K p at the planes of a slab needs p one plane below z0
  (the stress at z0 - 1 enters the backward-difference divergence) and one
  plane above z1 - 1 (the forward difference of the top plane); periodic
  across the first and last rank;
- an all-to-all transpose for the z transform of the preconditioner: the
  x-y transforms of each plane are local; the spectrum is then re-split
  from z-slabs into slabs of ky rows holding whole z lines, transformed and
  multiplied along z, and split back;
- an FP64 all-reduce of the two inner products <p, K p> and <r, M^-1 r>.
Nothing else crosses ranks.

This module holds the decomposition and the distributed PCG driver. The
per-slab arithmetic is passed in as a LocalOps object (the operator on a
slab with its halos, the x-y transforms of a slab's planes, the z
multiplier); the tests give it plain CPU tensor arithmetic and run the
ranks as gloo processes.
"""

import torch
import torch.distributed as dist


class SlabPlan:
    """Planes [z0, z1) of rank r (nz split as evenly as possible) and the ky
    rows [y0, y1) it holds in the transposed layout."""

    def __init__(self, nx, ny, nz, world, rank):
        self.nx, self.ny, self.nz, self.world, self.rank = nx, ny, nz, world, rank
        self.z_counts = [nz // world + (1 if r < nz % world else 0) for r in range(world)]
        self.y_counts = [ny // world + (1 if r < ny % world else 0) for r in range(world)]
        if min(self.z_counts) < 1 or min(self.y_counts) < 1:
            raise ValueError("every rank needs at least one z plane and one ky row")
        self.z0 = sum(self.z_counts[:rank])
        self.z1 = self.z0 + self.z_counts[rank]
        self.y0 = sum(self.y_counts[:rank])
        self.y1 = self.y0 + self.y_counts[rank]

    @property
    def nzl(self):
        return self.z1 - self.z0

    @property
    def nyl(self):
        return self.y1 - self.y0


def halo_exchange(x, plan, group=None):
    """x: (..., nzl + 2, ny, nx) with the slab in planes 1 .. nzl; fills
    plane 0 with the previous rank's top plane and plane nzl + 1 with the
    next rank's bottom plane (periodic). Real tensors."""
    world, rank = plan.world, plan.rank
    if world == 1:
        x[..., 0, :, :] = x[..., -2, :, :]
        x[..., -1, :, :] = x[..., 1, :, :]
        return x
    prev, nxt = (rank - 1) % world, (rank + 1) % world
    top = x[..., -2, :, :].contiguous()
    bottom = x[..., 1, :, :].contiguous()
    from_prev = torch.empty_like(top)
    from_next = torch.empty_like(bottom)
    reqs = [dist.isend(top, nxt, group=group), dist.isend(bottom, prev, group=group),
            dist.irecv(from_prev, prev, group=group), dist.irecv(from_next, nxt, group=group)]
    for q in reqs:
        q.wait()
    x[..., 0, :, :] = from_prev
    x[..., -1, :, :] = from_next
    return x


def _a2a(send_chunks, recv_shapes, dtype, group):
    """all_to_all_single of a list of per-rank chunks (real tensors)."""
    send = torch.cat([c.reshape(-1) for c in send_chunks]).contiguous()
    out_sizes = [int(torch.Size(s).numel()) for s in recv_shapes]
    recv = torch.empty(sum(out_sizes), dtype=dtype, device=send.device)
    dist.all_to_all_single(recv, send, output_split_sizes=out_sizes,
                           input_split_sizes=[c.numel() for c in send_chunks], group=group)
    return [t.reshape(s) for t, s in zip(recv.split(out_sizes), recv_shapes)]


def transpose_z_to_y(a, plan, group=None):
    """a: complex (C, nzl, ny, nx) in this rank's z-slab -> complex
    (C, nz, nyl, nx): every z plane of this rank's ky rows."""
    C = a.shape[0]
    ar = torch.view_as_real(a.contiguous())  # (C, nzl, ny, nx, 2)
    chunks = [ar[:, :, sum(plan.y_counts[:r]):sum(plan.y_counts[:r + 1])].contiguous() for r in range(plan.world)]
    shapes = [(C, plan.z_counts[r], plan.nyl, plan.nx, 2) for r in range(plan.world)]
    parts = _a2a(chunks, shapes, ar.dtype, group)
    return torch.view_as_complex(torch.cat(parts, dim=1).contiguous())


def transpose_y_to_z(b, plan, group=None):
    """Inverse of transpose_z_to_y: complex (C, nz, nyl, nx) -> (C, nzl, ny, nx)."""
    C = b.shape[0]
    br = torch.view_as_real(b.contiguous())  # (C, nz, nyl, nx, 2)
    chunks = [br[:, sum(plan.z_counts[:r]):sum(plan.z_counts[:r + 1])].contiguous() for r in range(plan.world)]
    shapes = [(C, plan.nzl, plan.y_counts[r], plan.nx, 2) for r in range(plan.world)]
    parts = _a2a(chunks, shapes, br.dtype, group)
    return torch.view_as_complex(torch.cat(parts, dim=2).contiguous())


def allreduce_sum(values, group=None):
    """FP64 sum over ranks of a list of local partial sums."""
    t = torch.tensor([float(v) for v in values], dtype=torch.float64)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, group=group)
    return [float(v) for v in t]


class LocalOps:
    """Per-slab arithmetic the driver needs (implemented by the caller).

    apply_K(p_halo) -> K p on the slab's planes, p_halo (D, nzl + 2, ny, nx)
      with its halo planes filled;
    residual(u_halo) -> f - K u on the slab's planes;
    fft_xy(x) / ifft_xy(X): 2D transforms of every plane (complex in/out);
    z_multiply(Y, plan): the z transform, the multiplier 1 / (m1 |D|^2) / N
      (0 at k = 0) and the inverse z transform of Y (C, nz, nyl, nx), whose
      rows are ky = plan.y0 .. plan.y1 - 1.
    """


def precondition(r, ops, plan, group=None):
    """z = M^-1 r on the slab (r: (D, nzl, ny, nx) real)."""
    R = ops.fft_xy(r.to(torch.complex128))
    Y = transpose_z_to_y(R, plan, group)
    Y = ops.z_multiply(Y, plan)
    Z = transpose_y_to_z(Y, plan, group)
    return ops.ifft_xy(Z).real


def slab_pcg(ops, plan, u0, tol=1e-12, max_iter=10000, group=None):
    """PCG on the slab-decomposed potential (the same iteration as the
    single-device solver: z = M^-1 r, beta = (r, z) / (r, z)_old,
    alpha = (r, z) / (p, K p); stop at sqrt((r, z) / (f, M^-1 f)) <= tol).
    u0: (D, nzl, ny, nx) float64 warm start. Returns (u, iterations,
    relative residual)."""
    D = u0.shape[0]
    shape_h = (D, plan.nzl + 2, plan.ny, plan.nx)
    u_h = torch.zeros(shape_h, dtype=torch.float64)
    u_h[:, 1:-1] = u0
    halo_exchange(u_h, plan, group)
    zero_h = torch.zeros(shape_h, dtype=torch.float64)
    f = ops.residual(zero_h)
    zf = precondition(f, ops, plan, group)
    (rz0,) = allreduce_sum([(f * zf).sum()], group)
    r = ops.residual(u_h)
    z = precondition(r, ops, plan, group)
    (rz,) = allreduce_sum([(r * z).sum()], group)
    if rz0 == 0.0:
        return u_h[:, 1:-1].clone(), 0, 0.0
    p_h = torch.zeros(shape_h, dtype=torch.float64)
    p_h[:, 1:-1] = z
    it = 0
    while rz > tol * tol * rz0 and it < max_iter:
        halo_exchange(p_h, plan, group)
        q = ops.apply_K(p_h)
        (pq,) = allreduce_sum([(p_h[:, 1:-1] * q).sum()], group)
        alpha = rz / pq
        u_h[:, 1:-1] += alpha * p_h[:, 1:-1]
        r = r - alpha * q
        z = precondition(r, ops, plan, group)
        (rz_new,) = allreduce_sum([(r * z).sum()], group)
        p_h[:, 1:-1] = z + (rz_new / rz) * p_h[:, 1:-1]
        rz = rz_new
        it += 1
    return u_h[:, 1:-1].clone(), it, (rz / rz0) ** 0.5
