"""CPU replay of a plan's operation list (test infrastructure).

Device buffers are numpy arrays filled with NaN; copies move planes; a kernel
op gathers its input planes and advances them `depth` steps with the FP64
oracle (on the sub-slab, whose outer planes the oracle holds fixed: those lie
outside the op's valid range, exactly like the trapezoid).  Ops execute one at
a time in a random order that respects only stream order and the op's
wait_op entries, so a missing cross-stream wait shows up as a wrong or NaN
result."""
import numpy as np

import oracle


def _new_planes(plan, o):
    """Planes the first launch of a chunk reads from the host grid in the
    zero-copy mode (run mode 3): the chunk's new planes of its round."""
    info = plan.info
    starts = plan.chunks()
    n0, r, T, k_off = info["dims"][0], info["radius"], info["time_steps"], info["k_off"]
    t, i = o["round"], o["chunk"]
    rounds = -(-T // k_off)
    kk = T % k_off if (t == rounds - 1 and T % k_off) else k_off
    s, e = starts[i], starts[i + 1]
    lo = 0 if i == 0 else min(n0, s + r * kk)
    hi = n0 if i == len(starts) - 2 else min(n0, e + r * kk)
    return lo, hi


def replay(plan, u0, coeff_fields=None, in_core=False, seed=0, policy="random"):
    info = plan.info
    nd = info["ndim"]
    shape = tuple(info["dims"][:nd])
    n0 = shape[0]
    pshape = shape[1:]
    r = info["radius"]
    kind = info["kind"]
    ops = plan.ops(in_core)
    bufs = plan.buffers(in_core)
    host = np.array(u0, dtype=np.float64, copy=True)
    dev = [np.full((max(cap, 0),) + pshape, np.nan) for _, cap in bufs]
    cdev = None
    if kind == 2:
        cdev = [np.full((6, max(cap, 0)) + pshape, np.nan) for _, cap in bufs]
    rng = np.random.default_rng(seed)

    def slots(slot0, n, cap):
        return (slot0 + np.arange(n)) % cap

    def run_op(o):
        k = o["kind"]
        if k == 0:  # host -> device
            lo, hi = o["src_lo"], o["src_hi"]
            b = o["dst_buf"]
            sl = slots(o["dst_slot0"], hi - lo, bufs[b][1])
            if kind == 2 and cdev is not None and _is_coef(o, in_core):
                cdev[b][:, sl] = coeff_fields[:, lo:hi]
            else:
                dev[b][sl] = host[lo:hi]
        elif k == 3:  # device -> device (region sharing of the result-reuse code)
            n = o["src_hi"] - o["src_lo"]
            sb, db = o["src_buf"], o["dst_buf"]
            dev[db][slots(o["dst_slot0"], n, bufs[db][1])] = dev[sb][slots(o["src_slot0"], n, bufs[sb][1])]
        elif k == 2:  # device -> host
            lo, hi = o["src_lo"], o["src_hi"]
            b = o["src_buf"]
            sl = slots(o["src_slot0"], hi - lo, bufs[b][1])
            host[o["dst_lo"]:o["dst_hi"]] = dev[b][sl]
        else:
            lo, hi = o["src_lo"], o["src_hi"]
            b = o["src_buf"]
            if int(in_core) == 3 and b == 0:
                # zero-copy input: the launch reads the chunk's new planes from
                # the host grid and writes them into the circular buffer
                nlo, nhi = _new_planes(plan, o)
                if nhi > nlo:
                    dev[0][slots(o["src_slot0"] + (nlo - lo), nhi - nlo, bufs[0][1])] = host[nlo:nhi]
            sub = dev[b][slots(o["src_slot0"], hi - lo, bufs[b][1])]
            depth = o["depth"]
            # the valid range of the last fused level must cover the output
            h = r * depth
            vlo = 0 if o["edge_lo"] else lo + h
            vhi = n0 if o["edge_hi"] else hi - h
            assert vlo <= o["dst_lo"] < o["dst_hi"] <= vhi, o
            assert (not o["edge_lo"] or lo == 0) and (not o["edge_hi"] or hi == n0), o
            if kind == 2:
                cb = 1
                cfs = cdev[cb][:, slots(_coef_slot0(o, plan, in_core, lo), hi - lo, bufs[cb][1])]
                res = oracle.run_varcoef(sub, cfs, depth)
            else:
                res = oracle.run(sub, plan._coeffs, r, kind, depth)
            out = res[o["dst_lo"] - lo:o["dst_hi"] - lo]
            db = o["dst_buf"]
            assert o["dst_hi"] - o["dst_lo"] <= bufs[db][1]
            dev[db][slots(o["dst_slot0"], o["dst_hi"] - o["dst_lo"], bufs[db][1])] = out

    # per-stream queues
    ns = 4
    queues = [[j for j, o in enumerate(ops) if o["stream"] == s] for s in range(ns)]
    pos = [0] * ns
    done = np.zeros(len(ops), dtype=bool)
    n_done = 0
    while n_done < len(ops):
        ready = []
        for s in range(ns):
            if pos[s] < len(queues[s]):
                j = queues[s][pos[s]]
                w = ops[j]["wait_op"]
                if all(w[t] < 0 or done[w[t]] for t in range(ns)):
                    ready.append(s)
        assert ready, "deadlock in the op list"
        if policy == "random":
            s = ready[rng.integers(len(ready))]
        elif policy == "h2d_first":
            s = min(ready)
        else:
            s = max(ready)
        j = queues[s][pos[s]]
        run_op(ops[j])
        done[j] = True
        pos[s] += 1
        n_done += 1
    return host


def _is_coef(o, in_core):
    return o["dst_buf"] == 1


def _coef_slot0(o, plan, in_core, lo):
    # the coefficient circular buffer shares the virtual plane indexing of the
    # input buffer: same capacity, same slot for a plane of the same round
    bufs = plan.buffers(in_core)
    if in_core:
        return lo
    cap = bufs[0][1]
    n0 = plan.info["dims"][0]
    return (o["round"] * n0 + lo) % cap
