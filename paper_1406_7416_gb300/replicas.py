"""Replica coordination for runs on several GPUs of one node.

The time step has no exchange step between independent grids, so several
GPUs run replicas: one process per GPU, each stepping its own grid, with no
collective on the data path (weak scaling).  The only collectives are a
barrier on each side of a timed region and a max-reduction of the elapsed
times: the slowest rank sets the job's time, and the job's rate is the units
all ranks processed divided by that time.

Launched by torchrun (RANK, LOCAL_RANK, WORLD_SIZE, MASTER_ADDR/PORT from the
environment); with WORLD_SIZE = 1 every call is local.  NCCL on GPUs, gloo on
CPU (the tests)."""
import os


class Replicas:
    def __init__(self, backend="nccl", device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            if backend == "nccl" and device is not None:
                dist.init_process_group(backend, device_id=device)
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max_over_ranks(self, x):
        """The largest value of `x` over the ranks (every rank gets it)."""
        if not self.dist:
            return float(x)
        import torch
        dev = self.device if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_rate(self, units_per_rank, seconds):
        """Units all ranks processed (each rank `units_per_rank`) per second of
        the slowest rank."""
        return units_per_rank * self.world / self.max_over_ranks(seconds)

    def close(self):
        if self.dist:
            self.dist.barrier()
            self.dist.destroy_process_group()
            self.dist = None
