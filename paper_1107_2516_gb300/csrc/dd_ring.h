// Host-side state of one served beam, with no device work: the sequence check
// a submission passes and the ring schedule a chunk follows when it runs.
// The server applies these steps to its device buffers; dd_server_ring_schedule
// runs them alone so that the schedule can be checked without a GPU.
#pragma once

#include <stdint.h>

#include "dd.h"

namespace dd {

// Submission order of one beam.  The first accepted chunk starts the stream;
// after it a chunk must carry the next sequence number (DD_OK).  A later
// number means chunks were lost: the chunk is accepted and restarts the
// stream (DD_SEQ_GAP).  A repeated or earlier number is refused (DD_ERR_SEQ):
// its samples belong before history the beam has already used.
struct SeqCheck {
    bool started = false;
    int64_t next = 0;

    int admit(int64_t seq, bool *restart)
    {
        *restart = false;
        if (!started) {
            started = true;
            next = seq + 1;
            return DD_OK;
        }
        if (seq == next) {
            next = seq + 1;
            return DD_OK;
        }
        if (seq < next) return DD_ERR_SEQ;
        *restart = true;
        next = seq + 1;
        return DD_SEQ_GAP;
    }
};

// Ring of `span` = maxshift + K*chunk columns per channel row.  A chunk is
// written at column `write` and de-dispersed from the window
// [write - maxshift, write + chunk) (Section 3, "Maximum shift": chunk outputs
// need chunk + maxshift inputs).  When the next chunk would pass `span`, the
// last maxshift samples move to columns [0, maxshift) first; with
// K = 2 + floor(maxshift / chunk) that happens at write = maxshift + K*chunk,
// so the move's source starts at K*chunk >= maxshift and never overlaps its
// destination.  The first chunks of a stream fill the history: a chunk is
// priming while fewer than maxshift real samples precede its window's end.
struct Ring {
    int64_t M = 0, chunk = 0, span = 0, write = 0, fed = 0;

    static int64_t span_of(int64_t maxshift, int64_t ch) { return maxshift + (2 + maxshift / ch) * ch; }

    void init(int64_t maxshift, int64_t ch)
    {
        M = maxshift;
        chunk = ch;
        span = span_of(maxshift, ch);
        write = maxshift;          // columns [0, maxshift) start as zeros
        fed = 0;
    }

    struct Step {
        bool zero_history;         // zero columns [0, maxshift) first (stream restart)
        int64_t move_src;          // >= 0: move columns [move_src, move_src + maxshift) to [0, maxshift)
        int64_t write_col;         // the chunk's first sample goes here
        int64_t window_col;        // the de-dispersion window starts here
        bool priming;              // no output yet
    };

    Step next(bool restart)
    {
        Step st{false, -1, 0, 0, false};
        if (restart) {
            st.zero_history = true;
            write = M;
            fed = 0;
        }
        if (write + chunk > span) {
            st.move_src = write - M;
            write = M;
        }
        st.write_col = write;
        st.window_col = write - M;
        st.priming = fed * chunk < M;
        write += chunk;
        ++fed;
        return st;
    }
};

}  // namespace dd
