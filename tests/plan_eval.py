"""Test-side numpy evaluation of an exported bucket schedule.

Checks the planner's structure (operands, masks, parents, roots) on the host,
without a GPU, by contracting the exported schedule with numpy in complex128
and comparing against the oracle. Leaf tensors are written out here from
their definitions (Eq. 2 gates), independently of the library's own leaf
kernel.
"""
import numpy as np


def leaf_tensor(kind: int, layer: int, gammas, betas) -> np.ndarray:
    """Entries [x + 2y] of a gate tensor (rank-1 tensors use [x])."""
    s = lambda x: 1 - 2 * x  # noqa: E731
    if kind == 0:  # |+>
        return np.array([1, 1, 0, 0], dtype=complex) / np.sqrt(2)
    if kind == 1:  # Z
        return np.array([1, -1, 0, 0], dtype=complex)
    T = np.zeros(4, dtype=complex)
    for x in (0, 1):
        for y in (0, 1):
            if kind in (2, 3):
                v = np.exp(-1j * gammas[layer] * s(x) * s(y))
            else:
                v = np.cos(betas[layer]) if x == y else -1j * np.sin(betas[layer])
            T[x + 2 * y] = np.conj(v) if kind in (3, 5) else v
    return T


def pext(o: np.ndarray, mask: int) -> np.ndarray:
    r = np.zeros_like(o)
    k = 0
    for bit in range(32):
        if (mask >> bit) & 1:
            r |= ((o >> bit) & 1) << k
            k += 1
    return r


def evaluate(buckets, operands, gammas, betas, graph_of_network=None, fixed=None):
    """Complex value of every network of the exported schedule.

    A sliced network's value is the sum over its slices of the product of the
    slice's root results and its fixed gate entries (`fixed`, from
    export_fixed); a gate with one variable fixed reads its entries from
    leaf_sub on."""
    n_nets = int(buckets["network"].max()) + 1
    res = {}
    sliced = "slice" in buckets.dtype.names
    slice_val = {}  # (network, slice) -> product
    for b in range(buckets.shape[0]):
        B = buckets[b]
        # a bucket sums n_sum variables (more than one: merged eliminations);
        # an operand's entry for output o and summed values s is
        # 2^popc(smask) * pext(o, mask) + pext(s, smask)
        n_sum = int(B["n_sum"]) if "n_sum" in B.dtype.names else 1
        n_out = int(B["width"]) - n_sum
        o = np.arange(1 << n_out, dtype=np.int64)
        acc = np.zeros(1 << n_out, dtype=complex)
        net = int(B["network"])
        g = 0 if graph_of_network is None else graph_of_network[net]
        gam = gammas[g] if np.ndim(gammas) == 2 else gammas
        bet = betas[g] if np.ndim(betas) == 2 else betas
        for x in range(1 << n_sum):
            prod = np.ones(1 << n_out, dtype=complex)
            for t in range(int(B["op_begin"]), int(B["op_begin"]) + int(B["n_ops"])):
                op = operands[t]
                sm = int(op["smask"]) if "smask" in op.dtype.names else 1
                idx = (pext(o, int(op["mask"])) << bin(sm).count("1")) + pext(np.int64(x), sm)
                if op["src"] < 0:
                    T = leaf_tensor(int(op["leaf_kind"]), int(op["leaf_layer"]), gam, bet)
                    if "leaf_sub" in op.dtype.names:
                        T = T[int(op["leaf_sub"]):]
                else:
                    T = res[int(op["src"])]
                prod = prod * T[idx]
            acc += prod
        res[b] = acc
        if B["parent"] < 0:
            key = (net, int(B["slice"]) if sliced else 0)
            slice_val[key] = slice_val.get(key, 1.0 + 0j) * acc[0]
    for f in (fixed if fixed is not None else []):
        net = int(f["network"])
        g = 0 if graph_of_network is None else graph_of_network[net]
        gam = gammas[g] if np.ndim(gammas) == 2 else gammas
        bet = betas[g] if np.ndim(betas) == 2 else betas
        key = (net, int(f["slice"]))
        slice_val[key] = slice_val[key] * leaf_tensor(int(f["leaf_kind"]), int(f["leaf_layer"]), gam, bet)[int(f["entry"])]
    value = np.zeros(n_nets, dtype=complex)
    for (net, _), v in slice_val.items():
        value[net] += v
    return value
