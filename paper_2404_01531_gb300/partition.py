"""Whole-instance partition of a batch of independent magnetospheres over
ranks (one process per GPU).

The instances of a batch share no data, so a batch splits over GPUs with no
exchange on the data path: each rank advances the instances it owns in its own
batched context, and only the timing and the counters are combined.  Work per
instance is estimated by its DG nodes, 6 n_ang^2 n_rad (P+1)^3 (the DG kernels
dominate a step and scale with the nodes; FD elements appear where the physics
puts them, unknown before the run).  The assignment is greedy
longest-processing-time: instances in decreasing work (ties by index) go to
the rank with the least work so far (ties to the lowest rank), so every rank
computes the same assignment from the same list of workloads."""


def instance_work(cfg):
    """Estimated work of one shell: its DG nodes."""
    return 6 * cfg["n_ang"] ** 2 * cfg["n_rad"] * (cfg["P"] + 1) ** 3


def assign_instances(cfgs, world):
    """owner[i] = the rank that advances instance i (0 <= owner < world)."""
    if world < 1:
        raise ValueError("world size must be at least 1")
    work = [instance_work(c) for c in cfgs]
    order = sorted(range(len(cfgs)), key=lambda i: (-work[i], i))
    loads = [0] * world
    owner = [0] * len(cfgs)
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        owner[i] = r
        loads[r] += work[i]
    return owner


def instances_of(cfgs, world, rank):
    """Indices of the instances rank `rank` owns, in increasing order."""
    owner = assign_instances(cfgs, world)
    return [i for i, r in enumerate(owner) if r == rank]
