"""Worker processes of the distributed tests (spawned; imported by the test files)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def gather_worker(rank, world, port, q):
    """Host side only: the all_gather helper over gloo with CPU tensors."""
    import torch
    import torch.distributed as dist
    from paper_1405_1931_gb300 import distributed as D
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    t = torch.arange(6, dtype=torch.int32) + 10 * rank
    got = D._all_gather(dist, None, t, on_device=False)
    n = torch.tensor([rank + 3], dtype=torch.int64)
    nn = D._all_gather(dist, None, n, on_device=False)
    q.put((rank, got.numpy(), nn.numpy()))
    dist.destroy_process_group()


def slab_worker(rank, world, port, cases, q):
    """Label this rank's slab of every case with label_slab over gloo on cuda:0."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1405_1931_gb300 import distributed as D
    from paper_1405_1931_gb300.hk import Labeller
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    lab = Labeller(0)
    out = []
    for phi, per in cases:
        nz = phi.shape[0]
        z0, nzr = D.slab_bounds(nz, world, rank)
        slab = torch.from_numpy(np.ascontiguousarray(phi[z0:z0 + nzr])).cuda()
        res = D.label_slab(lab, slab, z0, nz, per)
        torch.cuda.synchronize()
        out.append((z0, res.labels.cpu().numpy(), res.own_sizes.cpu().numpy(), res.offset, res.n_clusters,
                    res.hist.cpu().numpy()))
    lab.close()
    q.put((rank, out))
    dist.destroy_process_group()
