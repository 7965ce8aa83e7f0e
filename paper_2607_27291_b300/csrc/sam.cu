// sam.cu -- SAM text for drained hits (host code only).
//
// The paper streams headerless SAM records and writes the header (one @SQ
// line per contig) to a separate file, since the contig list is complete
// only at the end of the stream (Methods, "Output Format").  The primary
// record of a query is its first valid alignment in reference order
// (Results, accuracy validation); every later one is secondary (FLAG 256).
// Field readings are stated beside ifa_sam_records in ifa.h.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ifa.h"

namespace ifa {
void set_global_error(const std::string &msg);
}

namespace {

ifa_status sam_fail(const std::string &msg) {
    ifa::set_global_error(msg);
    return IFA_ERR_INVALID_ARG;
}

char upper_base(uint8_t c) {
    switch (c | 0x20) {
        case 'a': return 'A';
        case 'c': return 'C';
        case 'g': return 'G';
        case 't': return 'T';
        default: return 'N';
    }
}

char complement_base(uint8_t c) {
    switch (c | 0x20) {
        case 'a': return 'T';
        case 'c': return 'G';
        case 'g': return 'C';
        case 't': return 'A';
        default: return 'N';
    }
}

void append_u64(std::string &s, uint64_t v) {
    char buf[24];
    int n = 0;
    do {
        buf[n++] = static_cast<char>('0' + v % 10);
        v /= 10;
    } while (v);
    while (n) s.push_back(buf[--n]);
}

void append_name(std::string &s, const char *const *names, uint32_t n_names, uint32_t id, char prefix) {
    if (names && id < n_names && names[id]) {
        s.append(names[id]);
    } else {
        s.push_back(prefix);
        append_u64(s, id);
    }
}

ifa_status emit(const std::string &text, char *out, uint64_t cap, uint64_t *n_out) {
    *n_out = text.size();
    if (text.size() > cap) return sam_fail("ifa_sam: output buffer too small (" + std::to_string(text.size()) +
                                           " bytes needed)");
    if (!text.empty()) std::memcpy(out, text.data(), text.size());
    return IFA_OK;
}

}  // namespace

extern "C" {

ifa_status ifa_sam_records(ifa_hit *hits, uint64_t n, const ifa_sam_info *info, uint8_t *primary_seen,
                           char *out, uint64_t cap, uint64_t *n_out) {
    if (!info || !n_out || (n && !hits) || (cap && !out) || !primary_seen)
        return sam_fail("ifa_sam_records: null argument");
    if (!info->query_seqs || !info->query_lens) return sam_fail("ifa_sam_records: no query sequences");
    for (uint64_t i = 0; i < n; i++) {
        const ifa_hit &h = hits[i];
        if (h.query >= info->n_queries)
            return sam_fail("ifa_sam_records: hit names query " + std::to_string(h.query) + " of " +
                            std::to_string(info->n_queries));
        if (h.strand > 1) return sam_fail("ifa_sam_records: strand must be 0 or 1");
    }
    std::sort(hits, hits + n, [](const ifa_hit &a, const ifa_hit &b) {
        if (a.contig != b.contig) return a.contig < b.contig;
        if (a.pos != b.pos) return a.pos < b.pos;
        if (a.strand != b.strand) return a.strand < b.strand;
        if (a.query != b.query) return a.query < b.query;
        if (a.mismatches != b.mismatches) return a.mismatches < b.mismatches;
        return a.clips < b.clips;
    });
    // flags as they stand after this call; committed only if the text fits
    std::vector<uint8_t> seen(primary_seen, primary_seen + info->n_queries);
    std::string s;
    s.reserve(static_cast<size_t>(n) * 96);
    for (uint64_t i = 0; i < n; i++) {
        const ifa_hit &h = hits[i];
        const uint32_t L = info->query_lens[h.query];
        const uint8_t *q = info->query_seqs[h.query];
        if (!q && L) return sam_fail("ifa_sam_records: query " + std::to_string(h.query) + " has no sequence");
        const bool primary = !seen[h.query];
        seen[h.query] = 1;
        append_name(s, info->query_names, info->n_queries, h.query, 'q');
        s.push_back('\t');
        append_u64(s, (h.strand ? 16u : 0u) | (primary ? 0u : 256u));
        s.push_back('\t');
        append_name(s, info->contig_names, info->n_contig_names, h.contig, 'c');
        s.push_back('\t');
        append_u64(s, static_cast<uint64_t>(h.pos) + 1);
        s.append("\t255\t");
        const uint32_t left = h.clips & 0xffu, right = h.clips >> 8;
        if (left + right >= L && L) return sam_fail("ifa_sam_records: clips cover the whole query");
        if (left) {
            append_u64(s, left);
            s.push_back('S');
        }
        append_u64(s, L - left - right);
        s.push_back('M');
        if (right) {
            append_u64(s, right);
            s.push_back('S');
        }
        s.append("\t*\t0\t0\t");
        if (h.strand)
            for (uint32_t j = 0; j < L; j++) s.push_back(complement_base(q[L - 1 - j]));
        else
            for (uint32_t j = 0; j < L; j++) s.push_back(upper_base(q[j]));
        s.append("\t*\tNM:i:");
        append_u64(s, h.mismatches);
        s.push_back('\n');
    }
    const ifa_status st = emit(s, out, cap, n_out);
    if (st != IFA_OK) return st;
    std::memcpy(primary_seen, seen.data(), seen.size());
    return IFA_OK;
}

ifa_status ifa_sam_header(const char *const *contig_names, const uint32_t *contig_ids,
                          const uint64_t *contig_lens, uint32_t n, char *out, uint64_t cap, uint64_t *n_out) {
    if (!n_out || (n && !contig_lens) || (cap && !out)) return sam_fail("ifa_sam_header: null argument");
    if (n && !contig_names && !contig_ids) return sam_fail("ifa_sam_header: need contig names or ids");
    std::string s = "@HD\tVN:1.6\tSO:unsorted\n";
    for (uint32_t i = 0; i < n; i++) {
        s.append("@SQ\tSN:");
        if (contig_names && contig_names[i]) {
            s.append(contig_names[i]);
        } else {
            if (!contig_ids) return sam_fail("ifa_sam_header: contig " + std::to_string(i) + " has no name or id");
            s.push_back('c');
            append_u64(s, contig_ids[i]);
        }
        s.append("\tLN:");
        append_u64(s, contig_lens[i]);
        s.push_back('\n');
    }
    return emit(s, out, cap, n_out);
}

}  // extern "C"
