"""SAM text oracle -- TEST INFRASTRUCTURE ONLY.

Only the tests may import this module; the product path never does.

Plain restatement of the output the paper describes (Methods, "Output
Format"): headerless SAM records written as the stream goes, a separate
header listing the contigs, and the primary alignment of a query being its
first valid alignment in reference order (Results, accuracy validation).
The record fields follow the SAM format specification v1.6, section 1.4
(11 mandatory tab-separated fields, then optional TAG:TYPE:VALUE fields);
the values the paper leaves open take these readings: FLAG 0x10 for the
reverse strand and 0x100 for secondary records, MAPQ 255, CIGAR "<L>M", or
with soft clips at a contig end "<left>S<L - left - right>M<right>S" (the
SAM specification's soft clip, POS then being the first aligned base),
SEQ on the forward strand of the reference in upper case with non-ACGT
bytes written as N, QUAL "*", and the NM tag holding the mismatch count.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

_UPPER = {ord("A"): "A", ord("C"): "C", ord("G"): "G", ord("T"): "T"}
_COMPLEMENT = {"A": "T", "C": "G", "G": "C", "T": "A", "N": "N"}


def _forward_seq(q: bytes) -> str:
    return "".join(_UPPER.get(b & ~0x20, "N") for b in q)


def _reverse_complement(q: bytes) -> str:
    fwd = _forward_seq(q)
    return "".join(_COMPLEMENT[c] for c in reversed(fwd))


def sam_records(hits: Sequence[tuple], queries: Sequence[bytes], primary_seen: List[bool],
                query_names: Optional[Sequence[str]] = None,
                contig_names: Optional[Dict[int, str]] = None) -> str:
    """SAM lines for hits given as (query, contig, pos, strand, mismatches[,
    clips]) tuples, clips = left | right << 8.  `primary_seen[q]` is True
    once query q's primary was written; it is updated in place."""
    out = []
    hits = [tuple(h) + (0,) * (6 - len(h)) for h in hits]
    for (q, contig, pos, strand, mm, clips) in sorted(hits, key=lambda h: (h[1], h[2], h[3], h[0], h[4], h[5])):
        primary = not primary_seen[q]
        primary_seen[q] = True
        flag = 0
        if strand == 1:
            flag += 16
        if not primary:
            flag += 256
        qname = query_names[q] if query_names is not None else "q%d" % q
        rname = contig_names[contig] if contig_names is not None and contig in contig_names else "c%d" % contig
        seq = _reverse_complement(queries[q]) if strand == 1 else _forward_seq(queries[q])
        left, right = clips & 0xff, clips >> 8
        cigar = ("%dS" % left if left else "") + "%dM" % (len(queries[q]) - left - right) + \
            ("%dS" % right if right else "")
        fields = [qname, str(flag), rname, str(pos + 1), "255", cigar,
                  "*", "0", "0", seq, "*", "NM:i:%d" % mm]
        out.append("\t".join(fields) + "\n")
    return "".join(out)


def sam_header(contigs: Sequence[tuple]) -> str:
    """Header for (name, length) pairs, in the order given."""
    lines = ["@HD\tVN:1.6\tSO:unsorted\n"]
    for name, length in contigs:
        lines.append("@SQ\tSN:%s\tLN:%d\n" % (name, length))
    return "".join(lines)
