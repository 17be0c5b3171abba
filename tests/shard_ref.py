"""Reference joining of bucket-range builds for the tests (Section 5.2: the
ranges' node values and local offsets are concatenated, their Golomb-Rice
sequences joined bit after bit).  Plain numpy over the oracle's arrays;
shared by the CPU tests of the oracle's ranges and of the sharded driver."""
import numpy as np


def concat_bits(parts):
    """[(words, bits)] -> (words, bits) of the sequences one after another."""
    streams = [np.unpackbits(np.ascontiguousarray(w, np.uint64).view(np.uint8), bitorder="little")[:b]
               for w, b in parts]
    allb = np.concatenate(streams) if streams else np.zeros(0, np.uint8)
    total = int(allb.size)
    allb = np.concatenate([allb, np.zeros((-total) % 64, np.uint8)])
    return np.packbits(allb, bitorder="little").view(np.uint64), total


def concat_ranges(parts):
    """parts: per range, in bucket order, dicts with n, cum_keys, node_off,
    bit_pos (local, from 0), values, gr, gr_bits.  Returns the whole
    function's cum_keys, node_off, bit_pos, values, gr, gr_bits."""
    def offsets(name, base_key):
        out, base = [], 0
        for p in parts:
            out.append(np.asarray(p[name], np.uint64)[:-1] + np.uint64(base))
            base += int(p[base_key])
        out.append(np.array([base], np.uint64))
        return np.concatenate(out)

    gr, bits = concat_bits([(p["gr"], int(p["gr_bits"])) for p in parts])
    return {
        "cum_keys": offsets("cum_keys", "n"),
        "node_off": offsets("node_off", "n_nodes"),
        "bit_pos": offsets("bit_pos", "gr_bits"),
        "values": np.concatenate([np.asarray(p["values"], np.uint64) for p in parts]),
        "gr": gr,
        "gr_bits": bits,
    }


def oracle_part(o):
    return {"n": o.n, "cum_keys": o.cum_keys, "node_off": o.node_off, "bit_pos": o.bit_pos,
            "values": o.values, "gr": o.gr, "gr_bits": o.gr_bits, "n_nodes": o.n_nodes}


def bucket_of_keys(orc, keys, nb):
    hi, _ = orc.fingerprint(keys)
    return np.array([orc.bucket_of(int(h), nb) for h in hi], np.int64)
