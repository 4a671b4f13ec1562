"""Oracle: the integer FLOP and byte ledger of a sliced bucket-elimination schedule.

TEST INFRASTRUCTURE (see oracle/network.py).

The steps are those of Alg. 1 (bucket i: multiply its m tensors over the union
of their indices, rank u, and sum the bucket variable out, leaving rank
c = u - 1), with the execution reading of oracle/slicing.py: steps before the
first slice step run once on the unsliced network, later steps once per slice
on tensors whose sliced indices are fixed.

Per step, counted on complex numbers of `elem_bytes` bytes:
  flops = 6 (m - 1) 2^u + 2 (2^u - 2^c)   (complex multiply 6, complex add 2)
  bytes = elem_bytes * (sum over operands of 2^rank + 2^c)
(each operand read once, the result written once). The width of a step is c.
"""

from __future__ import annotations


def schedule_steps(tensor_labels, order, sliced=(), slice_step=0):
    """Symbolic bucket elimination: one record per processed bucket, in order."""
    sliced = set(sliced)
    pos = {v: i for i, v in enumerate(order)}
    nsteps = len(order)
    boundary = slice_step if sliced else 0
    buckets = [[] for _ in range(nsteps)]

    def earliest(labels):
        ranked = [pos[l] for l in labels if l in pos]
        return min(ranked) if ranked else None

    for labels in tensor_labels:
        e = earliest(labels)
        if e is not None:
            buckets[e].append(tuple(labels))
    steps = []
    for i in range(nsteps):
        bucket = buckets[i]
        if not bucket:
            continue
        region = "prefix" if i < boundary else "slice"
        v = order[i]
        if region == "slice":
            seen = [tuple(l for l in labels if l not in sliced) for labels in bucket]
        else:
            seen = bucket
        union = set()
        for labels in seen:
            union.update(labels)
        out_full = set()
        for labels in bucket:
            out_full.update(labels)
        out_full.discard(v)
        u = len(union)
        c = u - 1
        m = len(bucket)
        steps.append({
            "step": i, "var": v, "region": region, "m": m, "u": u, "c": c,
            "ranks": [len(l) for l in seen],
        })
        e = earliest(out_full)
        if e is not None:
            buckets[e].append(tuple(sorted(out_full)))
    return steps


def step_flops(m, u, c):
    return 6 * (m - 1) * (1 << u) + 2 * ((1 << u) - (1 << c))


def step_bytes(ranks, c, elem_bytes=8):
    return elem_bytes * (sum(1 << r for r in ranks) + (1 << c))


def ledger(tensor_labels, order, sliced=(), slice_step=0, elem_bytes=8):
    steps = schedule_steps(tensor_labels, order, sliced, slice_step)
    tot = {"prefix_flops": 0, "prefix_bytes": 0, "slice_flops": 0, "slice_bytes": 0,
           "prefix_width": 0, "slice_width": 0, "n_prefix_steps": 0, "n_slice_steps": 0}
    for st in steps:
        f = step_flops(st["m"], st["u"], st["c"])
        b = step_bytes(st["ranks"], st["c"], elem_bytes)
        st["flops"], st["bytes"] = f, b
        r = st["region"]
        tot[r + "_flops"] += f
        tot[r + "_bytes"] += b
        tot[r + "_width"] = max(tot[r + "_width"], st["c"])
        tot["n_" + r + "_steps"] += 1
    k = len(set(sliced))
    tot["k"] = k
    tot["total_flops"] = tot["prefix_flops"] + (tot["slice_flops"] << k)
    tot["total_bytes"] = tot["prefix_bytes"] + (tot["slice_bytes"] << k)
    return tot, steps


def launch_groups(tensor_labels, order, sliced=(), slice_step=0, max_nsum=6, max_ops=12,
                  elem_bytes=8):
    """Consecutive bucket steps grouped into one pass when their summed indices die together.

    Step j joins the group of step j-1 when: both are in the same region, the bucket
    vertex of j is the next position after that of j-1, the bucket of j holds the result
    of j-1, every other tensor of the bucket of j has all its (unsliced) indices inside
    the union U of the group's first step, the group then sums at most max_nsum indices
    and holds at most max_ops tensors. Such a group computes exactly the steps' products
    and sums (each step's own tensors multiplied in after the earlier indices are summed)
    without storing the intermediate results: its bytes are its tensors read once plus
    the last result written once; its flops are the sum of its steps' flops.
    """
    sliced_set = set(sliced)
    pos = {v: i for i, v in enumerate(order)}
    boundary = slice_step if sliced_set else 0

    def earliest(labels):
        ranked = [pos[l] for l in labels if l in pos]
        return min(ranked) if ranked else None

    # symbolic bucket elimination that keeps tensor identities
    buckets = [[] for _ in order]
    tensors = []  # labels of every tensor, gates first, then results in creation order
    for labels in tensor_labels:
        tensors.append(frozenset(labels))
        e = earliest(labels)
        if e is not None:
            buckets[e].append(len(tensors) - 1)
    steps = []
    for i, v in enumerate(order):
        if not buckets[i]:
            continue
        region = 0 if i < boundary else 1
        seen = {t: (tensors[t] if region == 0 else tensors[t] - sliced_set) for t in buckets[i]}
        union = frozenset().union(*seen.values())
        out = frozenset().union(*(tensors[t] for t in buckets[i])) - {v}
        tensors.append(out)
        rid = len(tensors) - 1
        m, u = len(buckets[i]), len(union)
        steps.append({"pos": i, "region": region, "ops": list(buckets[i]), "seen": seen,
                      "union": union, "out": rid,
                      "flops": step_flops(m, u, u - 1)})
        e = earliest(out)
        if e is not None:
            buckets[e].append(rid)
    groups = []
    for si, st in enumerate(steps):
        if groups:
            g = groups[-1]
            last = steps[g["first"] + g["nsteps"] - 1]
            others = [t for t in st["ops"] if t != last["out"]]
            if (st["region"] == g["region"] and st["pos"] == last["pos"] + 1
                    and last["out"] in st["ops"] and g["nsum"] + 1 <= max_nsum
                    and len(g["ops"]) + len(others) <= max_ops
                    and all(st["seen"][t] <= g["union"] for t in others)):
                g["nsteps"] += 1
                g["nsum"] += 1
                g["ops"] += [(t, st["seen"][t]) for t in others]
                g["flops"] += st["flops"]
                continue
        groups.append({"region": st["region"], "first": si, "nsteps": 1, "nsum": 1,
                       "union": st["union"], "flops": st["flops"],
                       "ops": [(t, st["seen"][t]) for t in st["ops"]]})
    out = []
    for g in groups:
        u = len(g["union"])
        c = u - g["nsum"]
        b = elem_bytes * (sum(1 << len(lab) for _, lab in g["ops"]) + (1 << c))
        out.append([g["region"], g["first"], g["nsteps"], len(g["ops"]), u, g["nsum"],
                    g["flops"], b])
    return out
